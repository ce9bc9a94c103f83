/*
 * iim.h -- C ABI of the GB300 immersed-interface Poisson solver.
 *
 * Solves  div(beta grad u) = f  on a uniform cell-centred grid of [-1,1]^d
 * (d = 2 or 3, n cells per axis, h = 2/n, node i at -1 + (i + 1/2) h) with an
 * immersed boundary or interface Gamma = {phi = 0} (Gabbard, Paris & van Rees,
 * "A high order multigrid-preconditioned immersed interface solver for the
 * Poisson equation with boundary and interface conditions", JCP 2025):
 *   Sec. 2.1, Eq. 1   boundary problems on Omega+ = {phi >= 0}:
 *                     u = ubar (Dirichlet) or beta+ du/dn = qbar (Neumann) on Gamma,
 *   Sec. 2.2, Eq. 8   interface problems: [u] = j0, [beta du/dn] = j1 on Gamma,
 * with n pointing out of Omega+ (towards Omega-) and [a] = a(+) - a(-).
 * The discretisation is the (n, n+1) IIM operator of Sec. 2.3 (Eq. 12): a 4th
 * or 6th order centred stencil with ghost values from least-squares
 * polynomials fitted at every control point (Eqs. 4-11).  The linear system
 * is solved by right-preconditioned FGMRES(m) (Sec. 4.1) with one
 * Shortley-Weller multigrid V-cycle as preconditioner (Sec. 3.1, 3.3).
 * An optional Dirichlet outer box closes the domain at the faces x_k = +-1.
 *
 * Memory and ownership
 *   Every pointer named *_dev is device memory owned by the caller and only
 *   borrowed for the duration of the call (asynchronous calls: until the work
 *   enqueued on the problem's stream has finished).  Every *_host pointer is
 *   host memory, borrowed likewise.  A problem owns its device workspace; it is
 *   allocated by iim_problem_create and released by iim_problem_destroy.
 *   Grid vectors are FP64, n^d entries, x0 fastest (flat index
 *   i0 + n i1 + n^2 i2).  Entries at nodes that are not unknowns (nodes of
 *   Omega- for boundary problems) are ignored on input and written as 0.
 *
 * Errors
 *   Every call returns an iim_status and never aborts; iim_last_error() gives
 *   a message for the calling thread.  Device-side failures are recorded in two
 *   status words on the device, one for the set-up (rank-deficient fits, the
 *   curvature bound, ...; cleared by every set-up) and one for the solve (NaN in
 *   the Krylov recurrence; cleared by every solve), and reported by the next call
 *   that synchronises (iim_problem_create, iim_solve, iim_status_get,
 *   iim_engine_release).  A problem stays usable after either kind of failure.
 */
#ifndef IIM_H
#define IIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IIM_OK = 0,
  IIM_ERR_INVALID_ARG = 1,   /* bad descriptor, option or pointer */
  IIM_ERR_CURVATURE = 2,     /* |kappa h| >= 1/4 at a control point (Sec. 2.1, Eq. 3) */
  IIM_ERR_RANK = 3,          /* least-squares fit rank deficient after growing its region */
  IIM_ERR_SINGULAR = 4,      /* Neumann s_c ~ 0 (Eq. 6) or interface denominator ~ 0 (Eq. 11) */
  IIM_ERR_NOT_CONVERGED = 5, /* FGMRES reached max_iter above tol */
  IIM_ERR_BREAKDOWN = 6,     /* NaN/Inf in the Krylov recurrence */
  IIM_ERR_BUDGET = 7,        /* device memory budget exceeded */
  IIM_ERR_TIMEOUT = 8,       /* a bounded device wait ran out */
  IIM_ERR_CUDA = 9,          /* CUDA runtime error */
  IIM_ERR_GEOMETRY = 10,     /* body too close to the outer box, or box missing */
  IIM_ERR_CAPACITY = 11      /* re-setup needs more workspace than allocated */
} iim_status;

enum { IIM_GEOM_CIRCLE = 0, IIM_GEOM_ELLIPSE = 1, IIM_GEOM_STAR = 2, IIM_GEOM_SPHERE = 3, IIM_GEOM_ELLIPSOID = 4,
       IIM_GEOM_PERTURBED_SPHERE = 5, IIM_GEOM_FOURIER = 6, IIM_GEOM_LEVELSET_GRID = 7 };
/* most modes of an IIM_GEOM_FOURIER curve */
enum { IIM_MAX_FOURIER_MODES = 16 };
enum { IIM_BC_DIRICHLET = 0, IIM_BC_NEUMANN = 1, IIM_BC_INTERFACE = 2 };
enum { IIM_BOX_NONE = 0, IIM_BOX_DIRICHLET = 1 };
/* Multigrid precision: FP32, FP64, or FP32 with every restricted residual (the
 * right-hand side of each coarser level) stored as 2-byte BF16 (rounded to nearest even)
 * and computed with in FP32. */
enum { IIM_MG_FP32 = 0, IIM_MG_FP64 = 1, IIM_MG_FP32_BF16R = 2 };
/* Multigrid cycle (Sec. 3.3 results): the V-cycle visits the next coarser level once
 * per visit of a level, the W-cycle twice, the second visit starting from the first
 * one's result with the same right-hand side. */
enum { IIM_CYCLE_V = 1, IIM_CYCLE_W = 2 };
/* Krylov method: right-preconditioned flexible GMRES(m) (Sec. 4.1), or left-
 * preconditioned GMRES(m) (Sec. 3.2), which minimises and tests the preconditioned
 * residual |M (b - A x)| <= tol |M b| and stores no preconditioned basis. */
enum { IIM_KRYLOV_FGMRES = 0, IIM_KRYLOV_GMRES_LEFT = 1 };

/* Problem statement (paper Sec. 2.1-2.2).
 * geom_params by kind (phi = -g if plus_inside else g, g < 0 inside the body):
 *   CIRCLE    cx cy R                 g = |x - c| - R
 *   ELLIPSE   cx cy a0 a1 angle       g = (y0/a0)^2 + (y1/a1)^2 - 1, y = Rot(-angle)(x - c)
 *   STAR      cx cy r0 amp m phase    g = |x - c| - (r0 + amp sin(m theta + phase))
 *   SPHERE    cx cy cz R
 *   ELLIPSOID cx cy cz a0 a1 a2       axis aligned
 *   PERTURBED_SPHERE cx cy cz rho0 rho1
 *                                     g = r - rho0 - rho1 Y(e), r = |x - c|, e = (x - c)/r,
 *                                     Y = (3 sqrt(3)/2) (e_x^2 - e_y^2) e_z (a degree-3 spherical
 *                                     harmonic scaled to max |Y| = 1; the radially perturbed
 *                                     sphere of the paper's 3D verification, Sec. 4.2)
 *   FOURIER   cx cy                   g = |x - c| - r(theta), r(theta) = a0 + sum_{k=1..K}
 *                                     (a_k cos k theta + b_k sin k theta): a closed curve given in
 *                                     parametric (polar) form, 2D.  The coefficients are in
 *                                     geom_coef; r must stay positive.  The coefficients are fixed
 *                                     at creation (iim_problem_setup may move the centre).
 *   LEVELSET_GRID (no parameters)     g = the level set given at the grid's own nodes (phi_dev),
 *                                     2D or 3D.  Between nodes g is the tensor product of the
 *                                     degree-5 Lagrange interpolants through the 6 nodes around
 *                                     the point along each axis (shifted inwards at the grid's
 *                                     edge), so that control points, normals (its gradient),
 *                                     curvatures (its Hessian) and the coarse multigrid levels
 *                                     all come from one function, exact for polynomial level
 *                                     sets of degree <= 5 in each variable.  This is the form
 *                                     of the paper's problem statement (Omega+ = {phi > 0},
 *                                     Sec. 2.1 and the level-set domain of Sec. 4.4) for shapes
 *                                     with no closed form here.  Needs n >= 16.
 */
typedef struct {
  int dim;               /* 2 or 3 */
  int n;                 /* cells per axis */
  int geom_kind;
  int plus_inside;       /* 1: Omega+ is the inside of the body */
  double geom_params[8];
  int bc;                /* IIM_BC_* */
  int box_bc;            /* IIM_BOX_*; interface problems need IIM_BOX_DIRICHLET */
  double beta_plus, beta_minus;
  int order;             /* 4 -> (4,5) scheme, 6 -> (6,7) scheme (Sec. 2.4) */
  /* IIM_GEOM_FOURIER: host array a0, a1, b1, ..., aK, bK (n_geom_coef = 2 K + 1, 1 <= K <=
   * IIM_MAX_FOURIER_MODES), copied by iim_problem_create.  NULL / 0 for other kinds. */
  const double* geom_coef;
  int n_geom_coef;
  /* IIM_GEOM_LEVELSET_GRID: device array of the level set at the n^dim nodes (x0 fastest),
   * copied by iim_problem_create (borrowed for that call only; iim_problem_set_phi replaces
   * the copy).  NULL for other kinds. */
  const double* phi_dev;
} iim_problem_desc;

typedef struct {
  double tol;            /* true relative residual |b - A x| / |b| (Sec. 4.3: 1e-10) */
  int restart;           /* FGMRES restart m (Sec. 4.1: 10), 1..16 */
  int max_iter;          /* total FGMRES iterations */
  int nu1, nu2;          /* pre/post red-black Gauss-Seidel sweeps */
  int mg_precision;      /* IIM_MG_FP32, IIM_MG_FP64 or IIM_MG_FP32_BF16R */
  int use_graph;         /* 1: the solve runs as one CUDA graph with device-side control */
  int reorth;            /* 1: second Gram-Schmidt pass when |w| drops below 1e-3 |w_old| */
  int cycle;             /* IIM_CYCLE_V or IIM_CYCLE_W (single-problem solves only) */
  int krylov;            /* IIM_KRYLOV_FGMRES or IIM_KRYLOV_GMRES_LEFT (single-problem solves only);
                            with GMRES_LEFT, tol and the reported relres are those of the
                            preconditioned residual */
} iim_options;

typedef struct {
  int status;            /* iim_status of the solve */
  int iters;             /* FGMRES iterations */
  int restarts;          /* completed restart cycles */
  int converged;
  double relres;         /* final true relative residual */
  double solve_ms;       /* device time of the solve */
  int64_t kernels;       /* kernels this solve executed on the device */
} iim_solve_info;

typedef struct iim_problem iim_problem;

/* Fill *opt with the defaults: tol 1e-10, restart 10, max_iter 500, V(2,2), FP32 MG, graph on,
 * reorth on, FGMRES. */
void iim_default_options(iim_options* opt);

/* Create a problem: validate, allocate the workspace and run the whole set-up
 * on the device (crossings, curvature check, least-squares fits, correction
 * records, Shortley-Weller levels, coarse LU).  ``stream`` is a cudaStream_t
 * (NULL = legacy default stream); all later work of this problem is enqueued
 * on it.  Synchronises.  On failure *out is NULL. */
iim_status iim_problem_create(const iim_problem_desc* desc, const iim_options* opt, void* stream,
                              iim_problem** out);

/* Re-run the set-up in place (same dim, n, bc, order, box), optionally with new
 * geometry parameters (params may be NULL).  Asynchronous: no allocation and no
 * host synchronisation; the workspace must be large enough (device-checked,
 * IIM_ERR_CAPACITY is reported by the next synchronising call).  With
 * opt.use_graph the set-up kernels are captured into a CUDA graph the first
 * time and replayed by later calls with the same geometry (new parameters
 * capture it again). */
iim_status iim_problem_setup(iim_problem* p, const double* geom_params);

/* Replace the level set of an IIM_GEOM_LEVELSET_GRID problem by phi_dev (n^dim values at
 * the grid's nodes, copied on the problem's stream); the next iim_problem_setup builds the
 * set-up from it.  IIM_ERR_INVALID_ARG for other geometry kinds.  Asynchronous. */
iim_status iim_problem_set_phi(iim_problem* p, const double* phi_dev);

/* Synchronise the problem's stream and return the device status word. */
iim_status iim_status_get(iim_problem* p);

void iim_problem_destroy(iim_problem* p);

/* Sizes: number of control points K, box data points B (2 d n^(d-1) or 0),
 * grid nodes N = n^d, unknowns. */
iim_status iim_problem_sizes(iim_problem* p, int* K, int* B, int64_t* N, int64_t* n_unknowns);

/* Device bytes the problem holds (its whole workspace). */
iim_status iim_problem_bytes(iim_problem* p, size_t* bytes);

/* Control points in canonical order (axis, then flat index of the lower node
 * of the cut grid edge): xc_dev [K][dim], normal_dev [K][dim] (out of Omega+).
 * Either pointer may be NULL.  Asynchronous. */
iim_status iim_control_points(iim_problem* p, double* xc_dev, double* normal_dev);

/* Grid edge of every control point, in the order of iim_control_points: axis_dev [K] the
 * axis of the cut edge, lower_dev [K] the flat index of its lower node, side_dev [K] 1 when
 * the lower node is in Omega+ (the edge leaves Omega+ in the + direction of the axis), else 0.
 * Any pointer may be NULL.  Asynchronous. */
iim_status iim_control_point_edges(iim_problem* p, int32_t* axis_dev, int32_t* lower_dev, uint8_t* side_dev);

/* Outer-box Dirichlet sample points (B of them, iim_problem_sizes): xb_dev [B][dim], in the
 * order iim_set_data takes box_dev: faces (-x0, +x0, -x1, +x1, -x2, +x2), within a face the
 * other node indices in flat order (lowest remaining axis fastest).  Each point lies on its
 * face (coordinate -1 or +1) with the other coordinates of its grid line, half a cell
 * beyond the line's last node.  IIM_ERR_INVALID_ARG without an outer box.  Asynchronous. */
iim_status iim_box_points(iim_problem* p, double* xb_dev);

/* Phase of every node (1 = Omega+) as bytes, n^d entries.  Asynchronous. */
iim_status iim_phase(iim_problem* p, uint8_t* phase_dev);

/* Data of Eq. 12 (L_Gamma u_Gamma): f_dev [N] source; g_dev [K] ubar (Dirichlet)
 * or qbar (Neumann); j0_dev, j1_dev [K] interface jumps; box_dev [B] outer-box
 * Dirichlet values, faces (-x0,+x0,-x1,+x1,-x2,+x2), each face flat over the
 * remaining node indices (lowest axis fastest).  Unused pointers may be NULL.
 * Computes b = f - L_Gamma u_Gamma on the device.  Asynchronous. */
iim_status iim_set_data(iim_problem* p, const double* f_dev, const double* g_dev, const double* j0_dev,
                        const double* j1_dev, const double* box_dev);

/* w = L_Omega u (+ L_Gamma u_Gamma of the last iim_set_data if include_data). Asynchronous. */
iim_status iim_apply(iim_problem* p, const double* u_dev, double* w_dev, int include_data);

/* The operator of iim_apply without touching the problem's own scratch.  The
 * paper has no counterpart: this is a deployment variant.  iim_apply writes the
 * ghost values into scratch that iim_problem_create allocated for that problem;
 * this call writes them into one fixed area compiled into the library (2^18
 * doubles = 2 MiB, reserved on every GPU that loads the library until the
 * process exits) and calls no cudaMalloc, cudaFree or allocating library
 * routine.  It is for callers that keep their problems' memory fixed once they
 * are set up and cannot allocate afterwards, such as code that runs under a hard
 * device-memory budget with nothing left to grow into.  The first call on a
 * device looks up the area's device address (with that device current); make
 * that first call before any stream capture begins.  Problems whose ghost
 * values exceed the area (2 x control points x w > 2^18 for interfaces, control
 * points x w otherwise) are rejected with IIM_ERR_CAPACITY before anything is
 * launched.  Every call shares the one area, which keeps the last call's
 * contents; each call writes every ghost value before reading it, so nothing
 * needs clearing, but calls that overlap on the device (other streams, threads
 * or problems) race and must be ordered by the caller.  Arguments and results
 * are those of iim_apply.  Asynchronous. */
iim_status iim_apply_noalloc(iim_problem* p, const double* u_dev, double* w_dev, int include_data);

/* b of the last iim_set_data.  Asynchronous. */
iim_status iim_rhs(iim_problem* p, double* b_dev);

/* z = one V-cycle of the Shortley-Weller multigrid applied to v / beta_sigma (Sec. 3.3). Asynchronous. */
iim_status iim_precondition(iim_problem* p, const double* v_dev, double* z_dev);

/* FGMRES solve of L_Omega x = b (Sec. 4.1).  x_dev: in x0, out x.  Synchronises. */
iim_status iim_solve(iim_problem* p, double* x_dev, iim_solve_info* info);

/* Same as iim_set_data + iim_solve with host buffers: copies f, g, j0, j1, box
 * host -> device, solves, and copies x back to x_host.  Synchronises. */
iim_status iim_solve_host(iim_problem* p, const double* f_host, const double* g_host, const double* j0_host,
                          const double* j1_host, const double* box_host, double* x_host, iim_solve_info* info);

/* Many independent problems (each created beforehand, each with its data set):
 * enqueues every solve graph on a pool of streams so that their kernels overlap
 * on the device, then waits.  infos may be NULL. */
iim_status iim_batch_solve(iim_problem** probs, double** x_devs, int count, iim_solve_info* infos);

/* ------------------------------------------------------------------------
 * Batched engine: many independent problems solved together.
 *
 * Each admitted problem ("slot") keeps its grids, multigrid hierarchy, Krylov
 * basis and FGMRES scalars on the device.  iim_engine_run launches one CUDA
 * graph that repeats a "tick" until every slot has finished or max_ticks ticks
 * have run; a tick advances every slot by one step of its own solve (an FGMRES
 * iteration of Sec. 4.1 with one V-cycle of Sec. 3.3, or a restart with the
 * true-residual test) through persistent kernels that walk device-side lists
 * of (slot, thread block) work items.  The work of a slot is split into the
 * same thread blocks as in iim_solve, so a slot's iterates, iteration count
 * and solution are bit for bit those of iim_solve on the same problem,
 * whatever else is in the engine.  Slots may be admitted and released between
 * runs; the lists are rewritten then, and the graph is captured again only
 * when a new kind of work appears.  The paper solves one problem at a time;
 * this batching is an addition of this library.
 *
 * All calls are on the engine's stream (stream argument of create; NULL = the
 * legacy default stream).  The engine only borrows problems: a problem must
 * stay alive until it is released, and must not be used by other calls while
 * admitted.
 * ---------------------------------------------------------------------- */
typedef struct iim_engine iim_engine;

/* Create an engine for up to max_slots problems solved with opt (tol, restart,
 * max_iter and reorth are taken per problem from the problem's own options;
 * nu1, nu2 and the FP32 multigrid are engine-wide: nu1, nu2 >= 2).  With
 * opt.use_graph = 0 a run enqueues the tick kernels one by one and reads the
 * unfinished-slot count after every tick (same results; for kernel profiling). */
iim_status iim_engine_create(const iim_options* opt, int max_slots, void* stream, iim_engine** out);
void iim_engine_destroy(iim_engine* e);

/* Admit a set-up problem whose data have been set (iim_set_data): its solve
 * starts at the next run from x0_dev (NULL: zero).  Work already enqueued on
 * the problem's stream comes first.  *slot receives the slot index.
 * IIM_ERR_CAPACITY when every slot is taken; IIM_ERR_INVALID_ARG when the
 * problem's multigrid options differ from the engine's. */
iim_status iim_engine_admit(iim_engine* e, iim_problem* p, const double* x0_dev, int* slot);

/* Enqueue one graph launch running up to max_ticks ticks (it stops earlier when
 * every slot has finished).  Asynchronous. */
iim_status iim_engine_run(iim_engine* e, int max_ticks);

/* Outcome of the last run: *live = slots still running, done[0 .. *ndone) =
 * slots that finished since the previous poll (done: int[max_slots]), and the
 * ticks run so far.  wait = 0 returns IIM_ERR_TIMEOUT at once while the run is
 * still on the device; wait = 1 blocks until it is done.  Any pointer may be NULL. */
iim_status iim_engine_poll(iim_engine* e, int wait, int* live, int* done, int* ndone, int64_t* ticks);

/* Remove a slot: copy its solution to x_dev (NULL: skip) and fill info (the
 * kernels field is 0: the engine's launches are shared, see iim_engine_stats).
 * Releasing a running slot cancels its solve (status IIM_ERR_TIMEOUT).
 * Synchronises the engine's stream. */
iim_status iim_engine_release(iim_engine* e, int slot, double* x_dev, iim_solve_info* info);

/* Kernel launches per tick of the captured graph, and ticks run so far. */
iim_status iim_engine_stats(iim_engine* e, int64_t* kernels_per_tick, int64_t* ticks);

/* Tile shapes of the fused 2D multigrid kernels per level size class (n <= 32,
 * 64, 128, 256, 512, larger; int[6]): 0 = 32x8, 1 = 64x8, 2 = 32x16, 3 = 64x16.
 * The shape changes the speed, not the result.  NULL restores the defaults. */
iim_status iim_engine_set_shapes(iim_engine* e, const int* shape_of_class);
iim_status iim_engine_get_shapes(iim_engine* e, int* shape_of_class);

/* Autotuner: for every size class in use, time the grouped V-cycle of all
 * admitted slots (reps repetitions) with each tile shape and keep the fastest;
 * *best_ms = the tuned V-cycle time.  It uses each slot's first Krylov vectors
 * as scratch, so it is only allowed before the first run after admission
 * (IIM_ERR_INVALID_ARG once a slot has started).  Synchronises. */
iim_status iim_engine_autotune(iim_engine* e, int reps, double* best_ms);

/* ------------------------------------------------------------------------
 * Request loop ("server") over an engine.
 *
 * Requests are queued by iim_server_submit and admitted, in submission order,
 * while the device memory they will hold fits hbm_budget bytes.  An admitted
 * request's problem is created and set up on its own stream by one of the
 * server's creation threads, beside the engine's work; the caller then sets its
 * data and marks it ready.  Ready
 * requests join the engine between runs of ticks_per_run ticks, and leave it
 * when their solve ends: their solution is copied to the host and their device
 * memory returned to the budget, so that queued requests can enter while
 * others are still running.  Nothing here blocks on the device except the
 * copy of a finished solution and iim_server_data_ready.  Latency of a
 * request: from iim_server_submit to its solution being on the host.
 * ---------------------------------------------------------------------- */
typedef struct iim_server iim_server;

/* opt as for iim_engine_create; max_slots problems on the device at once;
 * create_threads host threads create and set up admitted requests (1..64). */
iim_status iim_server_create(const iim_options* opt, size_t hbm_budget, int max_slots, int ticks_per_run,
                             int create_threads, iim_server** out);
/* Frees every request still held (running solves are cancelled). */
void iim_server_destroy(iim_server* s);

/* How admitted requests are solved (before the first submission): 0 = in the
 * batched engine, advanced together one FGMRES step per tick; 1 = each request's
 * own solve graph (captured by the creation thread) on its own stream, up to
 * max_slots at once, overlapping on the device.  Results are the same either way
 * and independent of the other requests. */
iim_status iim_server_set_mode(iim_server* s, int mode);

/* Reuse of retired problems (off by default): a finished request's problem (its allocation,
 * stream and solve graph) is kept, its bytes still counted against the budget, and a later
 * request of the same kind (dimension, n, conditions, outer box, order, geometry kind, side,
 * beta+, beta-; closed-form bodies only) takes it and re-runs its set-up in place with its own
 * geometry parameters, instead of creating a problem.  Kept problems are freed, oldest first,
 * when a new request needs their memory, or when reuse is switched off.  Results are those of
 * a fresh problem (the set-up leaves nothing of the earlier geometry behind).  Off by default:
 * serving streams with many reuses have stalled (kernels stopped completing on most streams,
 * one of them a reused problem's set-up), and the cause is not known. */
iim_status iim_server_set_pooling(iim_server* s, int on);
/* Requests that took a kept problem, requests created afresh, kept problems freed for room,
 * and problems kept now.  Any pointer may be NULL. */
iim_status iim_server_pool_stats(iim_server* s, int64_t* hits, int64_t* misses, int64_t* evicted, int* pooled);

/* Queue a request; *id identifies it.  IIM_ERR_BUDGET if it alone exceeds the budget. */
iim_status iim_server_submit(iim_server* s, const iim_problem_desc* desc, int64_t* id);

/* One turn of the loop: (1) when the last run has finished, release the slots
 * that finished; (2) put ready requests into free slots and launch the next run;
 * (3) copy the finished solutions to the host; (4) create queued requests that
 * fit the budget.  need_data[0 .. *n_need) = ids now waiting for data;
 * finished[0 .. *n_fin) = ids finished (or failed).  Every id is reported once:
 * ids beyond an array's capacity (or with a NULL array) are reported by a later step. */
iim_status iim_server_step(iim_server* s, int64_t* need_data, int cap_need, int* n_need, int64_t* finished,
                           int cap_fin, int* n_fin);

/* The problem of a request waiting for data (NULL otherwise): set its data with
 * iim_set_data (after iim_control_points / iim_phase as needed). */
iim_problem* iim_server_problem(iim_server* s, int64_t id);

/* The request's data are set: it joins the engine at the next run.  Waits for
 * the request's stream, so the caller's data buffers are free when it returns. */
iim_status iim_server_data_ready(iim_server* s, int64_t id);

/* End a request without a solution.  A queued request leaves the queue, and one waiting for
 * data or ready to run is freed, at once; one being created is freed when its creation ends;
 * a running one stops at the end of the engine's current run (mode 0) or when its solve graph
 * ends (mode 1: a graph launch is not interrupted).  The request is then reported finished
 * by a step, and iim_server_take returns IIM_ERR_TIMEOUT for it.  IIM_ERR_INVALID_ARG for an
 * unknown id or a request that has already ended.  Host only; does not wait. */
iim_status iim_server_cancel(iim_server* s, int64_t id);

/* Result of a finished request (x_host: n^d doubles, may be NULL), then forget
 * it.  Returns the request's final status; IIM_ERR_TIMEOUT while it is not finished. */
iim_status iim_server_take(iim_server* s, int64_t id, double* x_host, iim_solve_info* info, double* latency_s);

/* Device bytes held (or reserved) by requests now and at most so far, queued
 * requests, requests in the engine, engine runs launched, host seconds
 * (double[3], may be NULL): in iim_server_step, in copying solutions to the host,
 * and in creating requests (summed over the creation threads), and the number of
 * requests not yet taken in each state (int[8], may be NULL): queued, being
 * created, waiting for data, ready, running, retired, finished, failed.
 * Any pointer may be NULL. */
iim_status iim_server_stats(iim_server* s, size_t* bytes_in_use, size_t* peak_bytes, int* queued, int* resident,
                            int64_t* runs, double* host_seconds, int* states);

/* Boundary quantity the data do not prescribe, at every control point (K values,
 * the order of iim_control_points), from the same least-squares fits (Sec. 2.4):
 * Dirichlet problems: n . grad u(x_c) (n out of Omega+); Neumann problems: u(x_c)
 * (Eq. 6, with the qbar set by iim_set_data).  u_dev: n^d values (a solution).
 * Interface problems: IIM_ERR_INVALID_ARG.  Asynchronous. */
iim_status iim_boundary_values(iim_problem* p, const double* u_dev, double* out_dev);

/* grad u at every unknown node (Sec. 2.4): the centred first-derivative stencil of
 * the scheme's order (4 or 6) applied to the same extension of u as the operator
 * (u in its phase, the fits' ghost values with the problem's data past the first
 * control point, the outer-box ghosts).  grad_dev: dim x n^d values, axis-major
 * (component k of node i at k n^d + i); zero at nodes that are not unknowns.
 * Asynchronous. */
iim_status iim_gradient(iim_problem* p, const double* u_dev, double* grad_dev);

/* Profiling: average device time (microseconds) of one launch of an internal
 * kernel, timed with CUDA events on the problem's stream over ``reps`` back to
 * back launches on the problem's own vectors (after 3 untimed launches).
 * which: 0 high-order stencil, 1 ghost values, 2 corrections (Eq. 12 operator
 * kernels); 3 one red half sweep on the finest level; 4 FGMRES multi-dot and
 * 5 update over restart/2 + 1 vectors; 6 a whole V-cycle; 7 the whole operator;
 * 8 the least-squares fits of the set-up (Sec. 2.1-2.2); 9 / 10 the first level's fused
 * down / up multigrid kernel (2D, V(2,2); IIM_ERR_INVALID_ARG otherwise); 11 the coarse
 * single-CTA tail of the V-cycle.
 * Overwrites the problem's work vectors: call it between solves.  Synchronises. */
iim_status iim_kernel_time(iim_problem* p, int which, int reps, double* us);

/* The same, each timed launch alone and preceded by an overwrite of flush_dev
 * (flush_bytes of caller-owned device memory, larger than L2), so that the launch reads
 * its inputs from HBM.  flush_dev = NULL or flush_bytes = 0: as iim_kernel_time. */
iim_status iim_kernel_time_flushed(iim_problem* p, int which, int reps, void* flush_dev, size_t flush_bytes,
                                   double* us);

/* Least-squares fits of the current set-up: their number, the sum of their rows
 * (|X_c| + 1 each) and the monomial count M (for work estimates).  Synchronises. */
iim_status iim_problem_fit_stats(iim_problem* p, int64_t* nfit, int64_t* rows_sum, int* monomials);

/* Kernel launches issued by this library in the calling process so far. */
int64_t iim_launch_count(void);

const char* iim_last_error(void);
const char* iim_status_string(iim_status s);

#ifdef __cplusplus
}
#endif
#endif /* IIM_H */
