// Problem workspace and the entry points shared between the library's translation units.
#pragma once
#include <vector>

#include "common.cuh"

namespace iim {

// ---------------------------------------------------------------------------- device views
// Flat grid: node (i0, i1, i2) -> i0 + n i1 + n^2 i2.  Node coordinate x = -1 + (i + 1/2) h.
struct GridView {
  int dim, n;
  int64_t N;
  double h;
};

// One Shortley-Weller level (Sec. 3.1): aux[i] = -2 (not an unknown), -1 (regular
// unknown: standard 2d+1 point stencil), k >= 0 (irregular unknown, row k of the table).
// Table rows hold (diag, c[-x0], c[+x0], c[-x1], c[+x1], [c[-x2], c[+x2]]) of the
// homogeneous SW operator scaled by 1/h^2.
struct Level {
  GridView g;
  uint8_t* phase = nullptr;
  int32_t* aux = nullptr;
  uint8_t* cls = nullptr;         // per node: 1 unknown, 2 irregular row, 4 phase + (red-black tile kernels)
  int32_t* flag = nullptr;        // scratch for the irregular-node scan
  int32_t* idx = nullptr;
  int n_irr = 0, irr_cap = 0;
  int32_t* irr_node = nullptr;    // [irr_cap] node of each irregular row
  float* tab32 = nullptr;
  double* tab64 = nullptr;
  void* u = nullptr;              // level vectors, float or double by mg precision
  void* u2 = nullptr;             // second u buffer: fused kernels read one and write the other
  void* f = nullptr;
  int f_bf16 = 0;                 // the level's right-hand side (a restricted residual) is rounded to BF16
};

// device-side FGMRES state of one solve (krylov.cu)
struct SolverScalars {
  double H[(kMaxRestart + 1) * kMaxRestart];   // H[i + (kMaxRestart+1) * j]
  double g[kMaxRestart + 1];
  double cs[kMaxRestart], sn[kMaxRestart];
  double y[kMaxRestart];
  double inv_norm[kMaxRestart + 1];            // 1/|v_i| for the unnormalised basis
  double hcol[kMaxRestart + 2];
  double w2_old, w2;
  double bnorm, relres, est;
  int iters, restarts, k, active, done, converged, reorth_needed, breakdown;
  int m, max_iter, graph_mode, reorth;
  int first;                                   // batched engine: the next residual is the first
  double tol;
  cudaGraphConditionalHandle h_while;
  cudaGraphConditionalHandle h_if[kMaxRestart];
};

// parameters of the three operator kernels (operator.cu)
struct StencilCoef {
  double c0[2];            // d * a_0 * beta_sigma / h^2 for sigma = minus, plus
  double cj[2][kMaxW];     // a_j * beta_sigma / h^2
};

struct GhostParams {
  int nfit, w, rcap, bc, interface_, with_data;
  double beta_p, beta_m;
  const int* K;
  const int32_t* fit_R;
  const int32_t* fit_nodes;
  const double* fit_coef;
  const double* fit_cdat;
  const double* g;          // ubar / qbar per control point
  const double* j0;
  const double* j1;
  double* G;                // [nfit][w]
};

struct CorrectParams {
  GridView g;
  int w, q, with_data, n_aff_cap, nfit_cap;
  const int* n_aff;
  const int32_t* aff_node;
  const int32_t* aff_fit;
  const int32_t* aff_j;
  const double* G;
  const uint8_t* phase;
  const double* box;        // [B] face data
  double a[2 * kMaxW + 1];
  double scale[2];          // beta_sigma / h^2
  double box_w[kMaxW][8];
};

// slots of Problem::d_counts: control points, affected nodes, irregular rows of
// level l at kCountLevel0 + l (at most kMaxLevels levels), unknowns of the coarsest level
constexpr int kCountK = 0, kCountAff = 1, kCountLevel0 = 2, kMaxLevels = 24, kCountCoarse = 40, kCountSlots = 48;

struct Problem {
  iim_problem_desc desc;          // geom_coef and phi_dev are cleared after create (copies below)
  iim_options opt;
  std::vector<double> geom_coef;  // FOURIER coefficients
  double* phi_grid = nullptr;     // LEVELSET_GRID: the problem's copy of the node values
  cudaStream_t stream = nullptr;
  Geom geom;
  GridView g;
  int w = 0, q = 0, M = 0;        // stencil half width, fit degree, monomials
  double a[2 * kMaxW + 1];        // centred stencil a_{-w..w}
  int rcap = 0;                   // max least-squares rows per fit (excluding the control point)
  int box_active = 0;
  // fine grid
  uint8_t* phase = nullptr;       // 1 = Omega+
  // crossings / control points
  int32_t* edge_flag = nullptr;   // [dim * N]
  int32_t* edge_id = nullptr;     // [dim * N] exclusive scan -> crossing id of a cut edge
  int K = 0, K_cap = 0;
  int32_t* cr_edge = nullptr;     // [K_cap] cut edge (axis * N + lower node) of each control point
  int32_t* cr_axis = nullptr;
  int32_t* cr_lo = nullptr;
  uint8_t* cr_loplus = nullptr;
  double* cr_t = nullptr;
  double* cr_x = nullptr;         // [K][dim]
  double* cr_n = nullptr;         // [K][dim]
  double* cr_kappa = nullptr;
  // fits: boundary problems one per crossing (Omega+ side); interface two (2c: +, 2c+1: -)
  int nfit = 0, nfit_cap = 0;
  int32_t* fit_R = nullptr;       // [nfit]
  int* fit_overflow = nullptr;    // [nfit] fits the warp kernel hands to the CTA kernel
  int32_t* fit_nodes = nullptr;   // [nfit][rcap]
  double* fit_coef = nullptr;     // [nfit][w+1][rcap]
  double* fit_cdat = nullptr;     // [nfit][w+1]
  double* G = nullptr;            // [nfit][w] ghost values of the current apply
  int* d_monos = nullptr;         // [M][dim] exponents
  // affected nodes (nodes whose stencil meets a control point or the box)
  int32_t* aff_flag = nullptr;    // [N]
  int32_t* aff_idx = nullptr;     // [N]
  int n_aff = 0, aff_cap = 0;
  int32_t* aff_node = nullptr;    // [aff_cap]
  int32_t* aff_fit = nullptr;     // [aff_cap][2 dim]: fit id, -1 none, -2 box
  int32_t* aff_j = nullptr;       // [aff_cap][2 dim]: first out-of-phase offset jstar
  double box_w[kMaxW][8];         // box ghost Lagrange weights: [k][0] face, [k][m] node m+1
  // data (Eq. 12)
  double* d_g = nullptr;          // [K] ubar or qbar
  double* d_j0 = nullptr;
  double* d_j1 = nullptr;
  double* d_box = nullptr;        // [B]
  int B = 0;
  double* b = nullptr;            // right-hand side f - L_Gamma u_Gamma
  // Krylov
  double* V = nullptr;            // [(m+1)][Npad]
  double* Z = nullptr;            // [m][Npad]
  double* x = nullptr;
  double* tmp = nullptr;
  int64_t Npad = 0;
  SolverScalars* sc = nullptr;    // device
  double* partial = nullptr;      // [red_blocks][kMaxRestart + 4] reduction scratch
  unsigned int* counter = nullptr;
  int red_blocks = 0;
  // multigrid
  std::vector<Level> lv;
  int coarse_nu = 0;              // unknowns on the coarsest level at creation (sizes the LU's shared memory)
  int coarse_n = 0;               // size of the padded coarse system: the coarsest level's nodes (+1 when augmented)
  int aug = 0;                    // pure Neumann: the augmented system of Sec. 2.3 (one more unknown)
  int32_t* coarse_map = nullptr;  // [coarse_n] node of each slot of the coarse system, -1 if none
  double* coarse_lu64 = nullptr;  // [nu][nu] LU factors (row major), FP64
  float* coarse_lu32 = nullptr;
  int32_t* coarse_piv = nullptr;
  // status and scratch
  int* d_status = nullptr;
  int* d_counts = nullptr;        // [kCountSlots] device counters (see kCount*)
  int* scan_scratch = nullptr;
  int64_t scan_scratch_len = 0;
  // CUDA graph of the solve
  cudaGraphExec_t graph_exec = nullptr;
  int64_t kern_start = 0, kern_restart = 0, kern_iter[kMaxRestart] = {0};
  cudaGraph_t graph = nullptr;
  // CUDA graph of the set-up (geometry, fits, levels, coarse factor) for the current geometry
  cudaGraph_t setup_graph = nullptr;
  cudaGraphExec_t setup_exec = nullptr;
  int64_t kern_setup = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // a second stream for work that runs beside the main one (the ghost values beside the
  // stencil), joined back by events, also inside captured graphs
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  size_t bytes = 0;               // device bytes held
  std::vector<void*> allocs;
};

// scan.cu
int64_t scan_scratch_ints(int64_t len);
void scan_exclusive(const int* in, int* out, int64_t len, int* total, int* scratch, cudaStream_t s);

// setup.cu
iim_status setup_geometry(Problem& P, bool size_only);
iim_status setup_fits(Problem& P);
iim_status setup_levels(Problem& P, bool size_only);

// operator.cu
void ho_apply(Problem& P, const double* u, double* w, bool with_data, cudaStream_t s);
void ho_stencil(Problem& P, const double* u, double* w, cudaStream_t s);
void ho_ghost(Problem& P, const double* u, bool with_data, cudaStream_t s);
void ho_correct(Problem& P, const double* u, double* w, bool with_data, cudaStream_t s);
void box_points(Problem& P, double* xb, cudaStream_t s);
iim_status setup_direct(Problem& P, const double* params);
iim_status ho_apply_noalloc(Problem& P, const double* u, double* w, bool with_data, cudaStream_t s);
void compute_rhs(Problem& P, const double* f, cudaStream_t s);
iim_status boundary_values(Problem& P, const double* u, double* out, cudaStream_t s);
iim_status gradient(Problem& P, const double* u, double* grad, cudaStream_t s);
void eng_operator_params(Problem& P, StencilCoef* C, GhostParams* GP, CorrectParams* CP);

// multigrid.cu
void mg_precondition(Problem& P, const double* v, const double* vscale, double* z, cudaStream_t s);
bool mg_one_kernel(Problem& P, int which, const double* v, double* z, cudaStream_t s);
bool mg_has_fused_first(const Problem& P);
void mg_coarse_factor(Problem& P, cudaStream_t s);
void mg_smooth_fine(Problem& P, int colour, cudaStream_t s);

// krylov.cu
iim_status krylov_alloc(Problem& P);
void krylov_enqueue_solve(Problem& P, double* x, bool graph_mode);
iim_status krylov_build_graph(Problem& P, double* x);
void krylov_read_info(Problem& P, iim_solve_info* info);
void krylov_orth_pass(Problem& P, int j, int which, cudaStream_t s);

// api.cu
void* dev_alloc(Problem& P, size_t bytes);
iim_status solve_async(Problem& P);
iim_status solve_finish(Problem& P, iim_solve_info* info);
int rows_cap(int dim, int q);                  // least-squares rows reserved per fit
void set_error(const std::string& msg);

}  // namespace iim
