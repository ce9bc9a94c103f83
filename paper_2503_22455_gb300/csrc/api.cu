// C ABI of the library (declared in include/iim.h): problem life cycle, data,
// operator / preconditioner calls, the FGMRES solve and the batched solve.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "kernels.cuh"

namespace iim {

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

// Workspace comes from the device's stream-ordered memory pool, allocated and freed
// on the problem's stream: freeing a problem does not synchronise the device, so a
// request that finishes does not stall the solves still running.  The pool keeps
// freed memory for reuse (release threshold raised once per device).
static void keep_pool_memory() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  done[dev] = true;
}

void* dev_alloc(Problem& P, size_t bytes) {
  if (bytes == 0) bytes = 16;
  keep_pool_memory();
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, P.stream) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation failed for " + std::to_string(bytes) + " bytes");
    return nullptr;
  }
  P.allocs.push_back(p);
  P.bytes += bytes;
  return p;
}

// the problem's stream has finished every use of the workspace when this runs
static void free_all(Problem& P) {
  for (void* p : P.allocs) cudaFreeAsync(p, P.stream);
  P.allocs.clear();
  P.bytes = 0;
  if (P.graph_exec) cudaGraphExecDestroy(P.graph_exec);
  if (P.graph) cudaGraphDestroy(P.graph);
  if (P.setup_exec) cudaGraphExecDestroy(P.setup_exec);
  if (P.setup_graph) cudaGraphDestroy(P.setup_graph);
  P.setup_exec = nullptr;
  P.setup_graph = nullptr;
  if (P.ev0) cudaEventDestroy(P.ev0);
  if (P.ev1) cudaEventDestroy(P.ev1);
  if (P.ev_fork) cudaEventDestroy(P.ev_fork);
  if (P.ev_join) cudaEventDestroy(P.ev_join);
  if (P.side) cudaStreamDestroy(P.side);
  P.ev_fork = P.ev_join = nullptr;
  P.side = nullptr;
  P.graph_exec = nullptr;
  P.graph = nullptr;
  P.ev0 = nullptr;
  P.ev1 = nullptr;
}

static int binom(int a, int b) {
  int r = 1;
  for (int k = 1; k <= b; ++k) r = r * (a - b + k) / k;
  return r;
}

// centred second-derivative stencils a_{-w..w}: the unique symmetric stencils exact
// for polynomials of degree <= n+1 (Sec. 2.1; their sigma_max is Tab. 1)
static void stencil(int order, double* a) {
  if (order == 4) {
    const double h[3] = {-5.0 / 2.0, 4.0 / 3.0, -1.0 / 12.0};
    for (int j = -2; j <= 2; ++j) a[j + 2] = h[j < 0 ? -j : j];
  } else {
    const double h[4] = {-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0};
    for (int j = -3; j <= 3; ++j) a[j + 3] = h[j < 0 ? -j : j];
  }
}

// outer-box closure: Lagrange weights of the degree-q polynomial through the face
// value (position 0) and the nodes m = 2..q+1 from the face (positions -(m - 1/2)),
// evaluated at the ghosts k = 1..w (positions k - 1/2)
static void box_weights(int q, int w, double out[kMaxW][8]) {
  double pts[8];
  pts[0] = 0.0;
  for (int m = 2; m <= q + 1; ++m) pts[m - 1] = -(m - 0.5);
  for (int k = 0; k < kMaxW; ++k)
    for (int a = 0; a < 8; ++a) out[k][a] = 0.0;
  for (int k = 1; k <= w; ++k) {
    double x = k - 0.5;
    for (int a = 0; a <= q; ++a) {
      double num = 1, den = 1;
      for (int b = 0; b <= q; ++b)
        if (b != a) { num *= x - pts[b]; den *= pts[a] - pts[b]; }
      out[k - 1][a] = num / den;
    }
  }
}

// max rows of a least-squares set: lattice points of the half-ellipse (half
// ellipsoid) at the largest growth, with a one-cell margin on every semi-axis
int rows_cap(int dim, int q) {
  double an = q + 1.0 + 1.5 + 1.0, at = q / 2 + 1.0 + 1.5 + 1.0;
  double v = dim == 2 ? M_PI * an * at / 2.0 : 2.0 / 3.0 * M_PI * an * at * at;
  int cap = (int)std::ceil(v) + 8;
  return (cap + 7) / 8 * 8;
}

static std::vector<int> level_sizes(int n, int dim) {
  const int cmin = dim == 2 ? 8 : 4;
  std::vector<int> s{n};
  while (s.back() % 2 == 0 && s.back() / 2 >= cmin) s.push_back(s.back() / 2);
  return s;
}

static iim_status cuda_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return IIM_ERR_CUDA;
  }
  return IIM_OK;
}

static iim_status read_status(Problem& P) {
  int st[2] = {0, 0};
  if (cudaMemcpy(st, P.d_status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return cuda_check("status");
  if (st[0]) return (iim_status)st[0];
  return (iim_status)st[1];
}

static iim_status validate(const iim_problem_desc* d, const iim_options* o) {
  if (!d || !o) return IIM_ERR_INVALID_ARG;
  if (d->dim != 2 && d->dim != 3) return IIM_ERR_INVALID_ARG;
  if (d->order != 4 && d->order != 6) return IIM_ERR_INVALID_ARG;
  if (d->dim == 3 && d->order == 6) {
    set_error("3D problems support the (4,5) scheme");
    return IIM_ERR_INVALID_ARG;
  }
  if (d->n < 16 || d->n > (d->dim == 2 ? 32768 : 1024)) return IIM_ERR_INVALID_ARG;
  const bool grid = d->geom_kind == IIM_GEOM_LEVELSET_GRID;
  bool k2 = d->geom_kind == IIM_GEOM_CIRCLE || d->geom_kind == IIM_GEOM_ELLIPSE || d->geom_kind == IIM_GEOM_STAR ||
            d->geom_kind == IIM_GEOM_FOURIER || grid;
  bool k3 = d->geom_kind == IIM_GEOM_SPHERE || d->geom_kind == IIM_GEOM_ELLIPSOID ||
            d->geom_kind == IIM_GEOM_PERTURBED_SPHERE || grid;
  if ((d->dim == 2 && !k2) || (d->dim == 3 && !k3)) return IIM_ERR_INVALID_ARG;
  if (grid && !d->phi_dev) {
    set_error("a level set on the grid needs phi_dev");
    return IIM_ERR_INVALID_ARG;
  }
  if (d->geom_kind == IIM_GEOM_FOURIER) {
    const int nc = d->n_geom_coef;
    if (!d->geom_coef || nc < 3 || nc % 2 == 0 || nc > 2 * IIM_MAX_FOURIER_MODES + 1) {
      set_error("a Fourier curve needs 2 K + 1 coefficients, 1 <= K <= 16");
      return IIM_ERR_INVALID_ARG;
    }
    // r(theta) > 0 on a fine sampling of the curve
    double rmin = 1e300;
    for (int i = 0; i < 8192; ++i) {
      const double th = 6.283185307179586 * i / 8192.0;
      double r = d->geom_coef[0];
      for (int k = 1; 2 * k < nc; ++k) r += d->geom_coef[2 * k - 1] * std::cos(k * th) + d->geom_coef[2 * k] * std::sin(k * th);
      rmin = std::min(rmin, r);
    }
    if (!(rmin > 0)) {
      set_error("a Fourier curve needs r(theta) > 0");
      return IIM_ERR_INVALID_ARG;
    }
  }
  if (d->bc < 0 || d->bc > 2 || d->box_bc < 0 || d->box_bc > 1) return IIM_ERR_INVALID_ARG;
  if (d->bc == IIM_BC_INTERFACE && d->box_bc != IIM_BOX_DIRICHLET) {
    set_error("interface problems need a Dirichlet outer box");
    return IIM_ERR_INVALID_ARG;
  }
  if (!(d->beta_plus > 0) || (d->bc == IIM_BC_INTERFACE && !(d->beta_minus > 0))) return IIM_ERR_INVALID_ARG;
  if (o->restart < 1 || o->restart > kMaxRestart || o->max_iter < 1 || !(o->tol > 0)) return IIM_ERR_INVALID_ARG;
  if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 + o->nu2 < 1) return IIM_ERR_INVALID_ARG;
  if (o->mg_precision != IIM_MG_FP32 && o->mg_precision != IIM_MG_FP64 && o->mg_precision != IIM_MG_FP32_BF16R)
    return IIM_ERR_INVALID_ARG;
  if ((o->cycle != IIM_CYCLE_V && o->cycle != IIM_CYCLE_W) ||
      (o->krylov != IIM_KRYLOV_FGMRES && o->krylov != IIM_KRYLOV_GMRES_LEFT))
    return IIM_ERR_INVALID_ARG;
  return IIM_OK;
}

static int read_count(Problem& P, int k) {
  int v = 0;
  cudaMemcpyAsync(&v, P.d_counts + k, sizeof(int), cudaMemcpyDeviceToHost, P.stream);
  cudaStreamSynchronize(P.stream);
  return v;
}

size_t fit_smem_bytes(const Problem& P);

}  // namespace iim

using namespace iim;

struct iim_problem {
  Problem P;
};

extern "C" {

void iim_default_options(iim_options* o) {
  if (!o) return;
  o->tol = 1e-10;
  o->restart = 10;
  o->max_iter = 500;
  o->nu1 = 2;
  o->nu2 = 2;
  o->mg_precision = IIM_MG_FP32;
  o->use_graph = 1;
  o->reorth = 1;
  o->cycle = IIM_CYCLE_V;
  o->krylov = IIM_KRYLOV_FGMRES;
}

const char* iim_last_error(void) { return g_err.c_str(); }

const char* iim_status_string(iim_status s) {
  switch (s) {
    case IIM_OK: return "ok";
    case IIM_ERR_INVALID_ARG: return "invalid argument";
    case IIM_ERR_CURVATURE: return "curvature condition |kappa h| < 1/4 violated";
    case IIM_ERR_RANK: return "least-squares fit rank deficient";
    case IIM_ERR_SINGULAR: return "singular control-point closure";
    case IIM_ERR_NOT_CONVERGED: return "FGMRES did not converge";
    case IIM_ERR_BREAKDOWN: return "NaN/Inf in the Krylov recurrence";
    case IIM_ERR_BUDGET: return "device memory budget exceeded";
    case IIM_ERR_TIMEOUT: return "device wait timed out";
    case IIM_ERR_CUDA: return "CUDA error";
    case IIM_ERR_GEOMETRY: return "geometry too close to the outer box";
    case IIM_ERR_CAPACITY: return "workspace capacity exceeded";
  }
  return "unknown";
}

int64_t iim_launch_count(void) { return g_launches.load(); }

iim_status iim_problem_create(const iim_problem_desc* desc, const iim_options* opt, void* stream,
                              iim_problem** out) {
  if (!out) return IIM_ERR_INVALID_ARG;
  *out = nullptr;
  iim_status vs = validate(desc, opt);
  if (vs != IIM_OK) {
    if (g_err.empty()) set_error("invalid problem descriptor or options");
    return vs;
  }
  {
    cudaError_t stale = cudaGetLastError();
    if (stale != cudaSuccess) {
      set_error(std::string("error pending before create: ") + cudaGetErrorString(stale));
      return IIM_ERR_CUDA;
    }
  }
  iim_problem* H = new iim_problem();
  Problem& P = H->P;
  P.desc = *desc;
  P.opt = *opt;
  P.stream = (cudaStream_t)stream;
  if (desc->geom_kind == IIM_GEOM_FOURIER) P.geom_coef.assign(desc->geom_coef, desc->geom_coef + desc->n_geom_coef);
  P.desc.geom_coef = nullptr;
  P.desc.n_geom_coef = 0;
  P.desc.phi_dev = nullptr;
  const int d = desc->dim, n = desc->n;
  P.g.dim = d;
  P.g.n = n;
  P.g.N = (int64_t)n * n * (d == 3 ? n : 1);
  P.g.h = 2.0 / n;
  P.w = desc->order / 2;
  P.q = desc->order;
  P.M = binom(P.q + d, d);
  stencil(desc->order, P.a);
  P.rcap = rows_cap(d, P.q);
  P.box_active = desc->box_bc == IIM_BOX_DIRICHLET;
  P.B = P.box_active ? 2 * d * (int)(P.g.N / n) : 0;
  box_weights(P.q, P.w, P.box_w);
  const int64_t N = P.g.N;
  cudaEventCreate(&P.ev0);
  cudaEventCreate(&P.ev1);
  if (cudaStreamCreateWithFlags(&P.side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P.ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    P.side = nullptr;                  // no side stream: the operator runs its kernels in sequence
  }
  // monomials of total degree <= q, graded order
  std::vector<int> mono;
  for (int deg = 0; deg <= P.q; ++deg) {
    if (d == 2) {
      for (int a = deg; a >= 0; --a) { mono.push_back(a); mono.push_back(deg - a); mono.push_back(0); }
    } else {
      for (int a = deg; a >= 0; --a)
        for (int b = deg - a; b >= 0; --b) { mono.push_back(a); mono.push_back(b); mono.push_back(deg - a - b); }
    }
  }
  if (P.M > 40) { set_error("too many monomials"); free_all(P); delete H; return IIM_ERR_INVALID_ARG; }
#define IIM_FAIL(code) do { free_all(P); delete H; return (code); } while (0)
#define IIM_ALLOC(ptr, type, count)                                        \
  do {                                                                     \
    ptr = (type*)dev_alloc(P, sizeof(type) * (size_t)(count));             \
    if (!ptr) IIM_FAIL(IIM_ERR_BUDGET);                                    \
  } while (0)
  IIM_ALLOC(P.d_monos, int, mono.size());
  cudaMemcpyAsync(P.d_monos, mono.data(), sizeof(int) * mono.size(), cudaMemcpyHostToDevice, P.stream);
  cudaStreamSynchronize(P.stream);
  IIM_ALLOC(P.d_status, int, 4);
  if (desc->geom_kind == IIM_GEOM_LEVELSET_GRID) {
    IIM_ALLOC(P.phi_grid, double, N);
    if (cudaMemcpyAsync(P.phi_grid, desc->phi_dev, sizeof(double) * N, cudaMemcpyDeviceToDevice, P.stream) !=
        cudaSuccess) {
      cuda_check("copy of the level set");
      IIM_FAIL(IIM_ERR_INVALID_ARG);
    }
  }
  IIM_ALLOC(P.d_counts, int, kCountSlots);
  cudaMemsetAsync(P.d_status, 0, sizeof(int) * 4, P.stream);
  cudaMemsetAsync(P.d_counts, 0, sizeof(int) * kCountSlots, P.stream);
  IIM_ALLOC(P.phase, uint8_t, N);
  IIM_ALLOC(P.edge_flag, int32_t, N * d);
  IIM_ALLOC(P.edge_id, int32_t, N * d);
  IIM_ALLOC(P.aff_flag, int32_t, N);
  IIM_ALLOC(P.aff_idx, int32_t, N);
  P.scan_scratch_len = scan_scratch_ints(N * d) + 64;
  IIM_ALLOC(P.scan_scratch, int, P.scan_scratch_len);
  // pass 1: count crossings
  setup_geometry(P, true);
  int K = read_count(P, 0);
  if (cuda_check("setup: crossing count") != IIM_OK) IIM_FAIL(IIM_ERR_CUDA);
  P.K = K;
  P.K_cap = K + K / 4 + 64;
  IIM_ALLOC(P.cr_edge, int32_t, P.K_cap);
  IIM_ALLOC(P.cr_axis, int32_t, P.K_cap);
  IIM_ALLOC(P.cr_lo, int32_t, P.K_cap);
  IIM_ALLOC(P.cr_loplus, uint8_t, P.K_cap);
  IIM_ALLOC(P.cr_t, double, P.K_cap);
  IIM_ALLOC(P.cr_x, double, (size_t)P.K_cap * d);
  IIM_ALLOC(P.cr_n, double, (size_t)P.K_cap * d);
  IIM_ALLOC(P.cr_kappa, double, P.K_cap);
  cudaMemsetAsync(P.cr_kappa, 0, sizeof(double) * P.K_cap, P.stream);
  // pass 2: crossings, curvature, affected nodes
  setup_geometry(P, false);
  int n_aff = read_count(P, 1);
  if (cuda_check("setup: crossings") != IIM_OK) IIM_FAIL(IIM_ERR_CUDA);
  iim_status st = read_status(P);
  if (st != IIM_OK) {
    set_error(iim_status_string(st));
    IIM_FAIL(st);
  }
  P.n_aff = n_aff;
  P.aff_cap = n_aff + n_aff / 4 + 64;
  IIM_ALLOC(P.aff_node, int32_t, P.aff_cap);
  IIM_ALLOC(P.aff_fit, int32_t, (size_t)P.aff_cap * 2 * d);
  IIM_ALLOC(P.aff_j, int32_t, (size_t)P.aff_cap * 2 * d);
  const bool iface = desc->bc == IIM_BC_INTERFACE;
  P.nfit_cap = iface ? 2 * P.K_cap : P.K_cap;
  IIM_ALLOC(P.fit_R, int32_t, P.nfit_cap);
  IIM_ALLOC(P.fit_overflow, int, P.nfit_cap);
  IIM_ALLOC(P.fit_nodes, int32_t, (size_t)P.nfit_cap * P.rcap);
  IIM_ALLOC(P.fit_coef, double, (size_t)P.nfit_cap * (P.w + 1) * P.rcap);
  IIM_ALLOC(P.fit_cdat, double, (size_t)P.nfit_cap * (P.w + 1));
  IIM_ALLOC(P.G, double, (size_t)P.nfit_cap * P.w);
  cudaMemsetAsync(P.fit_R, 0, sizeof(int32_t) * P.nfit_cap, P.stream);
  if (fit_smem_bytes(P) > 227 * 1024) { set_error("least-squares workspace too large"); IIM_FAIL(IIM_ERR_INVALID_ARG); }
  st = setup_fits(P);
  if (st != IIM_OK) IIM_FAIL(st);
  cudaStreamSynchronize(P.stream);
  if (cuda_check("setup: fits") != IIM_OK) IIM_FAIL(IIM_ERR_CUDA);
  // data arrays
  IIM_ALLOC(P.d_g, double, P.K_cap);
  IIM_ALLOC(P.d_j0, double, P.K_cap);
  IIM_ALLOC(P.d_j1, double, P.K_cap);
  IIM_ALLOC(P.d_box, double, P.B > 0 ? P.B : 1);
  cudaMemsetAsync(P.d_g, 0, sizeof(double) * P.K_cap, P.stream);
  cudaMemsetAsync(P.d_j0, 0, sizeof(double) * P.K_cap, P.stream);
  cudaMemsetAsync(P.d_j1, 0, sizeof(double) * P.K_cap, P.stream);
  cudaMemsetAsync(P.d_box, 0, sizeof(double) * (P.B > 0 ? P.B : 1), P.stream);
  // pure Neumann: L 1 = 0; the solve runs on the augmented system [L 1; 1^T 0] (Sec. 2.3),
  // whose last entry (the shift alpha, the constraint gamma = 0) follows the grid vector
  P.aug = desc->bc == IIM_BC_NEUMANN && desc->box_bc == IIM_BOX_NONE;
  IIM_ALLOC(P.b, double, N + 1);
  cudaMemsetAsync(P.b, 0, sizeof(double) * (N + 1), P.stream);
  // multigrid levels
  std::vector<int> sizes = level_sizes(n, d);
  if ((int)sizes.size() > kMaxLevels) IIM_FAIL(IIM_ERR_INVALID_ARG);
  const size_t esz = opt->mg_precision == IIM_MG_FP64 ? 8 : 4;
  P.lv.resize(sizes.size());
  for (size_t l = 0; l < sizes.size(); ++l) {
    Level& L = P.lv[l];
    L.g.dim = d;
    L.g.n = sizes[l];
    L.g.N = (int64_t)sizes[l] * sizes[l] * (d == 3 ? sizes[l] : 1);
    L.g.h = 2.0 / sizes[l];
    L.f_bf16 = l > 0 && opt->mg_precision == IIM_MG_FP32_BF16R;
    if (l == 0) L.phase = P.phase;
    else IIM_ALLOC(L.phase, uint8_t, L.g.N);
    IIM_ALLOC(L.aux, int32_t, L.g.N);
    IIM_ALLOC(L.cls, uint8_t, L.g.N);
    IIM_ALLOC(L.flag, int32_t, L.g.N);
    IIM_ALLOC(L.idx, int32_t, L.g.N);
    L.u = dev_alloc(P, esz * L.g.N);
    L.u2 = dev_alloc(P, esz * L.g.N);
    const size_t fsz = L.f_bf16 ? 2 : esz;        // restricted residuals stored as BF16
    L.f = dev_alloc(P, fsz * L.g.N);
    if (!L.u || !L.u2 || !L.f) IIM_FAIL(IIM_ERR_BUDGET);
    cudaMemsetAsync(L.u, 0, esz * L.g.N, P.stream);
    cudaMemsetAsync(L.u2, 0, esz * L.g.N, P.stream);
    cudaMemsetAsync(L.f, 0, fsz * L.g.N, P.stream);
  }
  setup_levels(P, true);
  cudaStreamSynchronize(P.stream);
  if (cuda_check("setup: level classification") != IIM_OK) IIM_FAIL(IIM_ERR_CUDA);
  for (size_t l = 0; l < P.lv.size(); ++l) {
    Level& L = P.lv[l];
    L.n_irr = read_count(P, 2 + (int)l);
    L.irr_cap = L.n_irr + L.n_irr / 4 + 64;
    const int D = 2 * d + 1;
    IIM_ALLOC(L.irr_node, int32_t, L.irr_cap);
    IIM_ALLOC(L.tab64, double, (size_t)L.irr_cap * D);
    IIM_ALLOC(L.tab32, float, (size_t)L.irr_cap * D);
  }
  setup_levels(P, false);
  cudaStreamSynchronize(P.stream);
  if (cuda_check("setup: level tables") != IIM_OK) IIM_FAIL(IIM_ERR_CUDA);
  st = read_status(P);
  if (st != IIM_OK) { set_error(iim_status_string(st)); IIM_FAIL(st); }
  {
    // unknown count of the coarsest level from its aux codes (copied to the host once)
    Level& C = P.lv.back();
    std::vector<int32_t> aux(C.g.N);
    cudaMemcpy(aux.data(), C.aux, sizeof(int32_t) * C.g.N, cudaMemcpyDeviceToHost);
    int nu = 0;
    for (auto a : aux) nu += a != -2;
    if (C.g.N + P.aug > 4096) {
      set_error("the coarsest multigrid level has more than 4096 nodes: choose n with more factors of 2");
      IIM_FAIL(IIM_ERR_INVALID_ARG);
    }
    // the dense coarse system holds a slot per node of the coarsest level (+ the augmentation),
    // so that a later set-up with other geometry needs no other size
    P.coarse_nu = nu;
    P.coarse_n = (int)C.g.N + P.aug;
    const size_t cn = (size_t)P.coarse_n;
    IIM_ALLOC(P.coarse_map, int32_t, cn);
    IIM_ALLOC(P.coarse_piv, int32_t, cn > 0 ? cn : 1);
    IIM_ALLOC(P.coarse_lu64, double, 2 * cn * cn + 1);
    IIM_ALLOC(P.coarse_lu32, float, 2 * cn * cn + 1);
  }
  mg_coarse_factor(P, P.stream);
  cudaStreamSynchronize(P.stream);
  if (cuda_check("setup: coarse factor") != IIM_OK) IIM_FAIL(IIM_ERR_CUDA);
  if (krylov_alloc(P) != IIM_OK) IIM_FAIL(IIM_ERR_BUDGET);
  cudaStreamSynchronize(P.stream);
  st = read_status(P);
  if (st != IIM_OK) { set_error(iim_status_string(st)); IIM_FAIL(st); }
  if (cuda_check("create") != IIM_OK) IIM_FAIL(IIM_ERR_CUDA);
  *out = H;
  return IIM_OK;
#undef IIM_FAIL
#undef IIM_ALLOC
}

static iim_status setup_enqueue(Problem& P) {
  // the set-up status word reports this set-up alone (an earlier failed one is forgotten)
  cudaMemsetAsync(P.d_status, 0, sizeof(int), P.stream);
  setup_geometry(P, false);
  if (!(P.side && P.ev_fork && P.ev_join)) {
    iim_status st = setup_fits(P);
    if (st != IIM_OK) return st;
    setup_levels(P, false);
    mg_coarse_factor(P, P.stream);
    return IIM_OK;
  }
  // the Shortley-Weller levels and the coarse factor need the geometry but not the fits:
  // they run on the side stream beside the fits and are joined before the set-up ends
  cudaEventRecord(P.ev_fork, P.stream);
  cudaStreamWaitEvent(P.side, P.ev_fork, 0);
  const cudaStream_t main = P.stream;
  P.stream = P.side;
  setup_levels(P, false);
  mg_coarse_factor(P, P.stream);
  P.stream = main;
  cudaEventRecord(P.ev_join, P.side);
  const iim_status st = setup_fits(P);
  cudaStreamWaitEvent(P.stream, P.ev_join, 0);     // joined on every path
  return st;
}

// The set-up is a fixed sequence of kernels with no host decision in it, so (with
// use_graph) it is captured once per geometry and replayed as one graph launch.
}  // extern "C"

namespace iim {
// The set-up re-run in place with new geometry parameters, its kernels enqueued directly on the
// problem's stream (no graph capture; a captured set-up graph of other parameters is dropped).
// For the request loop's reuse of a retired problem.  Asynchronous.
iim_status setup_direct(Problem& P, const double* params) {
  bool changed = false;
  for (int k = 0; k < 8; ++k) {
    changed = changed || P.desc.geom_params[k] != params[k];
    P.desc.geom_params[k] = params[k];
  }
  if (changed && P.setup_exec) {
    cudaGraphExecDestroy(P.setup_exec);
    cudaGraphDestroy(P.setup_graph);
    P.setup_exec = nullptr;
    P.setup_graph = nullptr;
  }
  iim_status st = setup_enqueue(P);
  if (st != IIM_OK) return st;
  return cuda_check("setup");
}
}  // namespace iim

extern "C" {

iim_status iim_problem_set_phi(iim_problem* H, const double* phi_dev) {
  if (!H || !phi_dev) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  if (P.desc.geom_kind != IIM_GEOM_LEVELSET_GRID || !P.phi_grid) {
    set_error("iim_problem_set_phi: the problem's geometry is not a level set on the grid");
    return IIM_ERR_INVALID_ARG;
  }
  cudaMemcpyAsync(P.phi_grid, phi_dev, sizeof(double) * P.g.N, cudaMemcpyDeviceToDevice, P.stream);
  return cuda_check("iim_problem_set_phi");
}

iim_status iim_problem_setup(iim_problem* H, const double* params) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  if (params) {
    bool changed = false;
    for (int k = 0; k < 8; ++k) {
      changed = changed || P.desc.geom_params[k] != params[k];
      P.desc.geom_params[k] = params[k];
    }
    if (changed && P.setup_exec) {
      cudaGraphExecDestroy(P.setup_exec);
      cudaGraphDestroy(P.setup_graph);
      P.setup_exec = nullptr;
      P.setup_graph = nullptr;
    }
  }
  if (!P.opt.use_graph) {
    iim_status st = setup_enqueue(P);
    if (st != IIM_OK) return st;
    return cuda_check("setup");
  }
  if (!P.setup_exec) {
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return cuda_check("setup stream");
    cudaStream_t own = P.stream;
    P.stream = cs;
    cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    const int64_t c0 = iim_launch_count();
    iim_status st = setup_enqueue(P);
    P.kern_setup = iim_launch_count() - c0;
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(cs, &g);
    P.stream = own;
    cudaStreamDestroy(cs);
    if (st != IIM_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (cuda_check("setup capture") != IIM_OK || cudaGraphInstantiate(&P.setup_exec, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      P.setup_exec = nullptr;
      return cuda_check("setup graph");
    }
    P.setup_graph = g;
  }
  cudaGraphLaunch(P.setup_exec, P.stream);
  note_launches(P.kern_setup);
  return cuda_check("setup");
}

iim_status iim_status_get(iim_problem* H) {
  if (!H) return IIM_ERR_INVALID_ARG;
  cudaStreamSynchronize(H->P.stream);
  iim_status c = cuda_check("status");
  if (c != IIM_OK) return c;
  return read_status(H->P);
}

void iim_problem_destroy(iim_problem* H) {
  if (!H) return;
  cudaStreamSynchronize(H->P.stream);
  free_all(H->P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) fprintf(stderr, "iim_problem_destroy: CUDA error %s\n", cudaGetErrorString(e));
  delete H;
}

iim_status iim_problem_sizes(iim_problem* H, int* K, int* B, int64_t* N, int64_t* nunk) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  P.K = read_count(P, 0);
  if (K) *K = P.K;
  if (B) *B = P.B;
  if (N) *N = P.g.N;
  if (nunk) {
    if (P.desc.bc == IIM_BC_INTERFACE) *nunk = P.g.N;
    else {
      std::vector<uint8_t> ph(P.g.N);
      cudaMemcpy(ph.data(), P.phase, P.g.N, cudaMemcpyDeviceToHost);
      int64_t c = 0;
      for (auto v : ph) c += v;
      *nunk = c;
    }
  }
  return cuda_check("sizes");
}

iim_status iim_problem_bytes(iim_problem* H, size_t* bytes) {
  if (!H || !bytes) return IIM_ERR_INVALID_ARG;
  *bytes = H->P.bytes;
  return IIM_OK;
}

iim_status iim_problem_fit_stats(iim_problem* H, int64_t* nfit, int64_t* rows_sum, int* monomials) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  const int K = read_count(P, 0);
  const int nf = P.desc.bc == IIM_BC_INTERFACE ? 2 * K : K;
  std::vector<int32_t> R(nf > 0 ? nf : 1);
  if (nf > 0) cudaMemcpy(R.data(), P.fit_R, sizeof(int32_t) * nf, cudaMemcpyDeviceToHost);
  int64_t s = 0;
  for (int k = 0; k < nf; ++k) s += R[k] + 1;           // X_c plus the control point
  if (nfit) *nfit = nf;
  if (rows_sum) *rows_sum = s;
  if (monomials) *monomials = P.M;
  return cuda_check("fit stats");
}

iim_status iim_control_points(iim_problem* H, double* xc, double* nrm) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  int K = P.K = read_count(P, 0);
  if (xc) cudaMemcpyAsync(xc, P.cr_x, sizeof(double) * (size_t)K * P.g.dim, cudaMemcpyDeviceToDevice, P.stream);
  if (nrm) cudaMemcpyAsync(nrm, P.cr_n, sizeof(double) * (size_t)K * P.g.dim, cudaMemcpyDeviceToDevice, P.stream);
  return cuda_check("control points");
}

iim_status iim_control_point_edges(iim_problem* H, int32_t* axis, int32_t* lower, uint8_t* side) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  int K = P.K = read_count(P, 0);
  if (axis) cudaMemcpyAsync(axis, P.cr_axis, sizeof(int32_t) * (size_t)K, cudaMemcpyDeviceToDevice, P.stream);
  if (lower) cudaMemcpyAsync(lower, P.cr_lo, sizeof(int32_t) * (size_t)K, cudaMemcpyDeviceToDevice, P.stream);
  if (side) cudaMemcpyAsync(side, P.cr_loplus, (size_t)K, cudaMemcpyDeviceToDevice, P.stream);
  return cuda_check("control point edges");
}

iim_status iim_box_points(iim_problem* H, double* xb) {
  if (!H || !xb) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  if (!P.box_active) {
    set_error("iim_box_points: the problem has no outer box");
    return IIM_ERR_INVALID_ARG;
  }
  box_points(P, xb, P.stream);
  return cuda_check("box points");
}

iim_status iim_phase(iim_problem* H, uint8_t* phase) {
  if (!H || !phase) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  cudaMemcpyAsync(phase, P.phase, P.g.N, cudaMemcpyDeviceToDevice, P.stream);
  return cuda_check("phase");
}

// K (the control-point count) is the count of the last set-up whose size the
// host has read (create, iim_problem_sizes, iim_control_points)
static void copy_data(Problem& P, const double* g, const double* j0, const double* j1, const double* box,
                      cudaMemcpyKind kind) {
  const int Kn = P.K;
  if (g) cudaMemcpyAsync(P.d_g, g, sizeof(double) * Kn, kind, P.stream);
  if (j0) cudaMemcpyAsync(P.d_j0, j0, sizeof(double) * Kn, kind, P.stream);
  if (j1) cudaMemcpyAsync(P.d_j1, j1, sizeof(double) * Kn, kind, P.stream);
  if (box && P.B > 0) cudaMemcpyAsync(P.d_box, box, sizeof(double) * P.B, kind, P.stream);
}

iim_status iim_set_data(iim_problem* H, const double* f, const double* g, const double* j0, const double* j1,
                        const double* box) {
  if (!H || !f) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  copy_data(P, g, j0, j1, box, cudaMemcpyDeviceToDevice);
  compute_rhs(P, f, P.stream);
  return cuda_check("set_data");
}

iim_status iim_apply(iim_problem* H, const double* u, double* w, int include_data) {
  if (!H || !u || !w) return IIM_ERR_INVALID_ARG;
  ho_apply(H->P, u, w, include_data != 0, H->P.stream);
  return cuda_check("apply");
}

iim_status iim_apply_noalloc(iim_problem* H, const double* u, double* w, int include_data) {
  if (!H || !u || !w) return IIM_ERR_INVALID_ARG;
  iim_status st = ho_apply_noalloc(H->P, u, w, include_data != 0, H->P.stream);
  if (st != IIM_OK) return st;
  return cuda_check("apply_noalloc");
}

iim_status iim_boundary_values(iim_problem* H, const double* u, double* out) {
  if (!H || !u || !out) return IIM_ERR_INVALID_ARG;
  iim_status st = boundary_values(H->P, u, out, H->P.stream);
  if (st != IIM_OK) return st;
  return cuda_check("boundary values");
}

iim_status iim_gradient(iim_problem* H, const double* u, double* grad) {
  if (!H || !u || !grad) return IIM_ERR_INVALID_ARG;
  iim_status st = gradient(H->P, u, grad, H->P.stream);
  if (st != IIM_OK) return st;
  return cuda_check("gradient");
}

iim_status iim_rhs(iim_problem* H, double* b) {
  if (!H || !b) return IIM_ERR_INVALID_ARG;
  cudaMemcpyAsync(b, H->P.b, sizeof(double) * H->P.g.N, cudaMemcpyDeviceToDevice, H->P.stream);
  return cuda_check("rhs");
}

iim_status iim_precondition(iim_problem* H, const double* v, double* z) {
  if (!H || !v || !z) return IIM_ERR_INVALID_ARG;
  mg_precondition(H->P, v, nullptr, z, H->P.stream);
  return cuda_check("precondition");
}

static iim_status solve_enqueue(Problem& P, cudaStream_t s) {
  if (P.opt.use_graph) {
    if (!P.graph_exec) {
      iim_status st = krylov_build_graph(P, P.x);
      if (st != IIM_OK) return st;
    }
    cudaMemsetAsync(P.d_status + 1, 0, sizeof(int), s);
    cudaGraphLaunch(P.graph_exec, s);
    note_launch();
  } else {
    cudaMemsetAsync(P.d_status + 1, 0, sizeof(int), s);
    krylov_enqueue_solve(P, P.x, false);
  }
  return cuda_check("solve");
}

static iim_status finish_info(Problem& P, iim_solve_info* info) {
  iim_solve_info tmp;
  std::memset(&tmp, 0, sizeof(tmp));
  krylov_read_info(P, &tmp);
  float ms = 0;
  cudaEventElapsedTime(&ms, P.ev0, P.ev1);
  tmp.solve_ms = ms;
  iim_status st = read_status(P);
  if (st == IIM_OK && !tmp.converged) st = IIM_ERR_NOT_CONVERGED;
  tmp.status = st;
  if (info) *info = tmp;
  if (st != IIM_OK) set_error(iim_status_string(st));
  return st;
}

}  // extern "C"

namespace iim {
// asynchronous solve of the problem's own data from x = 0 on its stream (request loop)
iim_status solve_async(Problem& P) {
  cudaMemsetAsync(P.x, 0, sizeof(double) * (P.g.N + P.aug), P.stream);
  cudaEventRecord(P.ev0, P.stream);
  iim_status st = solve_enqueue(P, P.stream);
  cudaEventRecord(P.ev1, P.stream);
  return st;
}
iim_status solve_finish(Problem& P, iim_solve_info* info) {
  cudaStreamSynchronize(P.stream);
  if (cuda_check("solve") != IIM_OK) return IIM_ERR_CUDA;
  return finish_info(P, info);
}
}  // namespace iim

extern "C" {

iim_status iim_solve(iim_problem* H, double* x, iim_solve_info* info) {
  if (!H || !x) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  cudaMemcpyAsync(P.x, x, sizeof(double) * P.g.N, cudaMemcpyDeviceToDevice, P.stream);
  if (P.aug) cudaMemsetAsync(P.x + P.g.N, 0, sizeof(double), P.stream);   // alpha starts at 0
  cudaEventRecord(P.ev0, P.stream);
  const int64_t l0 = iim_launch_count();
  iim_status st = solve_enqueue(P, P.stream);
  if (st != IIM_OK) return st;
  const int64_t l1 = iim_launch_count();
  cudaEventRecord(P.ev1, P.stream);
  cudaMemcpyAsync(x, P.x, sizeof(double) * P.g.N, cudaMemcpyDeviceToDevice, P.stream);
  cudaStreamSynchronize(P.stream);
  if (cuda_check("solve") != IIM_OK) return IIM_ERR_CUDA;
  iim_solve_info tmp;
  st = finish_info(P, &tmp);
  if (!P.opt.use_graph) tmp.kernels = l1 - l0;
  if (info) *info = tmp;
  return st;
}

iim_status iim_solve_host(iim_problem* H, const double* f, const double* g, const double* j0, const double* j1,
                          const double* box, double* x, iim_solve_info* info) {
  if (!H || !f || !x) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  // stage f in the last Krylov basis vector, which the solve overwrites only later
  double* fst = P.V + (size_t)P.opt.restart * P.Npad;
  cudaMemcpyAsync(fst, f, sizeof(double) * P.g.N, cudaMemcpyHostToDevice, P.stream);
  copy_data(P, g, j0, j1, box, cudaMemcpyHostToDevice);
  compute_rhs(P, fst, P.stream);
  cudaMemsetAsync(P.x, 0, sizeof(double) * (P.g.N + P.aug), P.stream);
  cudaEventRecord(P.ev0, P.stream);
  const int64_t l0 = iim_launch_count();
  iim_status st = solve_enqueue(P, P.stream);
  if (st != IIM_OK) return st;
  const int64_t l1 = iim_launch_count();
  cudaEventRecord(P.ev1, P.stream);
  cudaMemcpyAsync(x, P.x, sizeof(double) * P.g.N, cudaMemcpyDeviceToHost, P.stream);
  cudaStreamSynchronize(P.stream);
  if (cuda_check("solve_host") != IIM_OK) return IIM_ERR_CUDA;
  iim_solve_info tmp;
  st = finish_info(P, &tmp);
  if (!P.opt.use_graph) tmp.kernels = l1 - l0;
  if (info) *info = tmp;
  return st;
}

iim_status iim_batch_solve(iim_problem** probs, double** xs, int count, iim_solve_info* infos) {
  if (count < 0 || (count > 0 && (!probs || !xs))) return IIM_ERR_INVALID_ARG;
  static std::mutex mu;
  static std::vector<cudaStream_t> pool;
  static std::vector<cudaEvent_t> evs;
  {
    std::lock_guard<std::mutex> lk(mu);
    while ((int)pool.size() < 16) {
      cudaStream_t s;
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      pool.push_back(s);
    }
    while ((int)evs.size() < count) {
      cudaEvent_t e;
      cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      evs.push_back(e);
    }
  }
  iim_status worst = IIM_OK;
  for (int i = 0; i < count; ++i) {
    Problem& P = probs[i]->P;
    if (P.opt.use_graph && !P.graph_exec) {
      iim_status st = krylov_build_graph(P, P.x);
      if (st != IIM_OK) return st;
    }
  }
  for (int i = 0; i < count; ++i) {
    Problem& P = probs[i]->P;
    cudaStream_t s = pool[i % pool.size()];
    cudaEventRecord(evs[i], P.stream);
    cudaStreamWaitEvent(s, evs[i], 0);
    cudaMemcpyAsync(P.x, xs[i], sizeof(double) * P.g.N, cudaMemcpyDeviceToDevice, s);
    if (P.aug) cudaMemsetAsync(P.x + P.g.N, 0, sizeof(double), s);
    cudaEventRecord(P.ev0, s);
    cudaMemsetAsync(P.d_status + 1, 0, sizeof(int), s);
    if (P.opt.use_graph) {
      cudaGraphLaunch(P.graph_exec, s);
      note_launch();
    }
    cudaEventRecord(P.ev1, s);
    cudaMemcpyAsync(xs[i], P.x, sizeof(double) * P.g.N, cudaMemcpyDeviceToDevice, s);
  }
  for (size_t k = 0; k < pool.size(); ++k) cudaStreamSynchronize(pool[k]);
  if (cuda_check("batch") != IIM_OK) return IIM_ERR_CUDA;
  for (int i = 0; i < count; ++i) {
    Problem& P = probs[i]->P;
    if (!P.opt.use_graph) {
      cudaMemcpy(P.x, xs[i], sizeof(double) * P.g.N, cudaMemcpyDeviceToDevice);
      if (P.aug) cudaMemset(P.x + P.g.N, 0, sizeof(double));
      cudaMemsetAsync(P.d_status + 1, 0, sizeof(int), P.stream);
      krylov_enqueue_solve(P, P.x, false);
      cudaMemcpyAsync(xs[i], P.x, sizeof(double) * P.g.N, cudaMemcpyDeviceToDevice, P.stream);
      cudaStreamSynchronize(P.stream);
    }
    iim_status st = finish_info(P, infos ? &infos[i] : nullptr);
    if (st != IIM_OK && worst == IIM_OK) worst = st;
  }
  return worst;
}

iim_status iim_kernel_time_flushed(iim_problem* H, int which, int reps, void* flush, size_t flush_bytes, double* us) {
  if (!H || !us || reps < 1) return IIM_ERR_INVALID_ARG;
  Problem& P = H->P;
  cudaStream_t s = P.stream;
  const int j = P.opt.restart / 2;
  auto launch = [&]() {
    switch (which) {
      case 0: ho_stencil(P, P.x, P.tmp, s); break;
      case 1: ho_ghost(P, P.x, false, s); break;
      case 2: ho_correct(P, P.x, P.tmp, false, s); break;
      case 3: mg_smooth_fine(P, 0, s); break;
      case 4: krylov_orth_pass(P, j, 0, s); break;
      case 5: krylov_orth_pass(P, j, 1, s); break;
      case 6: mg_precondition(P, P.V, nullptr, P.tmp, s); break;
      case 7: ho_apply(P, P.x, P.tmp, false, s); break;
      case 8: setup_fits(P); break;
      case 9: mg_one_kernel(P, 0, P.V, P.tmp, s); break;
      case 10: mg_one_kernel(P, 1, P.V, P.tmp, s); break;
      case 11: mg_one_kernel(P, 2, P.V, P.tmp, s); break;
      default: break;
    }
  };
  if (which < 0 || which > 11) return IIM_ERR_INVALID_ARG;
  if (which >= 9 && which <= 10 && !mg_has_fused_first(P)) {
    set_error("kernel_time: the problem has no fused first-level multigrid kernels");
    return IIM_ERR_INVALID_ARG;
  }
  for (int r = 0; r < 3; ++r) launch();
  if (flush && flush_bytes > 0) {
    // each launch alone after overwriting a buffer larger than L2: its inputs come from HBM
    double tot = 0;
    for (int r = 0; r < reps; ++r) {
      cudaMemsetAsync(flush, r & 0xff, flush_bytes, s);
      cudaEventRecord(P.ev0, s);
      launch();
      cudaEventRecord(P.ev1, s);
      cudaEventSynchronize(P.ev1);
      float ms = 0;
      cudaEventElapsedTime(&ms, P.ev0, P.ev1);
      tot += ms;
    }
    *us = 1e3 * tot / reps;
    return cuda_check("kernel time");
  }
  cudaEventRecord(P.ev0, s);
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(P.ev1, s);
  cudaEventSynchronize(P.ev1);
  float ms = 0;
  cudaEventElapsedTime(&ms, P.ev0, P.ev1);
  *us = 1e3 * ms / reps;
  return cuda_check("kernel time");
}

iim_status iim_kernel_time(iim_problem* H, int which, int reps, double* us) {
  return iim_kernel_time_flushed(H, which, reps, nullptr, 0, us);
}

}  // extern "C"
