// The (n, n+1) IIM operator w = L_Omega u (+ L_Gamma u_Gamma), paper Sec. 2.3, Eq. 12.
//
// Split into three kernels:
//   k_ho_stencil  every unknown node: beta_sigma/h^2 sum_axes sum_j a_j u_{i+j e}, where
//                 neighbours outside phase sigma (or outside the box) contribute 0;
//   k_ho_ghost    one warp per control point: u_c (Dirichlet data, Neumann elimination
//                 Eqs. 5-6, or the interface closure Eqs. 9-11) and the w ghost values
//                 p_c(x_g) = s_c u_c + sum s_a u_a of Eq. 4;
//   k_ho_correct  one thread per affected node: adds a_j p_c(x_{i+j e}) for every
//                 out-of-phase offset past the first control point of each walk, and
//                 the outer-box ghosts.
// The stencil is FP64 and bound by the FP64 pipe on GB300 (2 FMA/clk/SM), so it
// is written to use the fewest FP64 operations: neighbours at equal |j| are
// summed first, then one FMA per |j| with beta/h^2 folded into the coefficients.
#include <mutex>
#include <string>

#include "engine.cuh"

namespace iim {


template <int D, int W>
__device__ __forceinline__ void ho_stencil_node(const GridView& g, const StencilCoef& C, int interface_,
                                                const double* __restrict__ u, const uint8_t* __restrict__ phase,
                                                double* __restrict__ w, int64_t i) {
  const int n = g.n;
  const uint8_t ph = phase[i];
  if (!interface_ && !ph) { w[i] = 0.0; return; }
  int m[3];
  m[0] = (int)(i % n);
  int64_t r = i / n;
  m[1] = (int)(r % n);
  m[2] = D > 2 ? (int)(r / n) : 0;
  const int sig = ph ? 1 : 0;
  double acc = C.c0[sig] * u[i];
#pragma unroll
  for (int j = 1; j <= W; ++j) {
    double v[2 * D];
#pragma unroll
    for (int ax = 0; ax < D; ++ax) {
      const int64_t st = ax == 0 ? 1 : (ax == 1 ? (int64_t)n : (int64_t)n * n);
      v[2 * ax] = 0.0;
      v[2 * ax + 1] = 0.0;
      if (m[ax] - j >= 0) {
        int64_t nb = i - j * st;
        double t = u[nb];
        v[2 * ax] = phase[nb] == ph ? t : 0.0;
      }
      if (m[ax] + j < n) {
        int64_t nb = i + j * st;
        double t = u[nb];
        v[2 * ax + 1] = phase[nb] == ph ? t : 0.0;
      }
    }
    double s = v[0];
#pragma unroll
    for (int k = 1; k < 2 * D; ++k) s += v[k];
    acc = fma(C.cj[sig][j - 1], s, acc);
  }
  w[i] = acc;
}

template <int D, int W>
__global__ void __launch_bounds__(256) k_ho_stencil(GridView g, StencilCoef C, int interface_,
                                                    const double* __restrict__ u,
                                                    const uint8_t* __restrict__ phase, double* __restrict__ w) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  ho_stencil_node<D, W>(g, C, interface_, u, phase, w, i);
}


// Eight lanes per control point: each lane accumulates an eighth of the X_c terms
// of every row (sequential FMAs, no per-term reduction), then two shuffle steps
// combine the quarters.  Boundary problems: rows 0..w-1 of fit c.  Interface
// problems: rows 0..w of fits 2c (+) and 2c+1 (-), then the closure of Eqs. 9-11.
constexpr int kGhostLanes = 8;

__device__ inline double quad_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4, kGhostLanes);
  v += __shfl_xor_sync(0xffffffffu, v, 2, kGhostLanes);
  v += __shfl_xor_sync(0xffffffffu, v, 1, kGhostLanes);
  return v;
}

template <int W>
__device__ __forceinline__ void ho_ghost_body(const GhostParams& P, const double* __restrict__ u, int gid) {
  const int c = gid / kGhostLanes, q = gid % kGhostLanes;
  const int K = *P.K;
  const bool live = c < K;                       // every lane takes part in the shuffles
  const int rows = W + 1;
  const int nsides = P.interface_ ? 2 : 1;
  double acc[2][W + 1];
#pragma unroll
  for (int sd = 0; sd < 2; ++sd)
#pragma unroll
    for (int k = 0; k <= W; ++k) acc[sd][k] = 0.0;
#pragma unroll
  for (int sd = 0; sd < 2; ++sd) {
    if (sd >= nsides || !live) continue;
    const int f = P.interface_ ? 2 * c + sd : c;
    const int R = P.fit_R[f];
    const int32_t* nodes = P.fit_nodes + (size_t)f * P.rcap;
    const double* coef = P.fit_coef + (size_t)f * rows * P.rcap;
    const int nr = P.interface_ ? W + 1 : W;
    for (int a = q; a < R; a += kGhostLanes) {
      const double ua = u[nodes[a]];
#pragma unroll
      for (int k = 0; k <= W; ++k)
        if (k < nr) acc[sd][k] = fma(coef[(size_t)k * P.rcap + a], ua, acc[sd][k]);
    }
  }
#pragma unroll
  for (int sd = 0; sd < 2; ++sd)
#pragma unroll
    for (int k = 0; k <= W; ++k)
      if (sd < nsides) acc[sd][k] = quad_sum(acc[sd][k]);
  if (!live || q != 0) return;
  if (!P.interface_) {
    const double data = P.with_data ? P.g[c] : 0.0;
#pragma unroll
    for (int k = 0; k < W; ++k) P.G[(size_t)c * W + k] = acc[0][k] + P.fit_cdat[(size_t)c * rows + k] * data;
    return;
  }
  // Eqs. 9-11: S = b+ s+_c - b- s-_c ; ubar = -(b+ D+ - b- D-)/S
  const double *cp = P.fit_cdat + (size_t)(2 * c) * rows, *cm = P.fit_cdat + (size_t)(2 * c + 1) * rows;
  const double bp = P.beta_p, bm = P.beta_m;
  const double Sden = bp * cp[W] - bm * cm[W];
  const double ubar = -(bp * acc[0][W] - bm * acc[1][W]) / Sden;
  double up = ubar, um = ubar;
  if (P.with_data) {
    up = ubar + (P.j1[c] - bm * cm[W] * P.j0[c]) / Sden;
    um = ubar + (P.j1[c] - bp * cp[W] * P.j0[c]) / Sden;
  }
#pragma unroll
  for (int k = 0; k < W; ++k) {
    P.G[(size_t)(2 * c) * W + k] = acc[0][k] + cp[k] * up;
    P.G[(size_t)(2 * c + 1) * W + k] = acc[1][k] + cm[k] * um;
  }
}

template <int W>
__global__ void __launch_bounds__(256) k_ho_ghost(GhostParams P, const double* __restrict__ u) {
  ho_ghost_body<W>(P, u, blockIdx.x * blockDim.x + threadIdx.x);
}


__device__ __forceinline__ void ho_correct_body(const CorrectParams& P, const double* __restrict__ u,
                                                double* __restrict__ w, int t) {
  if (t >= *P.n_aff || t >= P.n_aff_cap) return;
  const GridView& g = P.g;
  const int n = g.n, d = g.dim, W = P.w;
  const int64_t i = P.aff_node[t];
  int m[3];
  m[0] = (int)(i % n);
  int64_t r = i / n;
  m[1] = (int)(r % n);
  m[2] = d > 2 ? (int)(r / n) : 0;
  const uint8_t ph = P.phase[i];
  double acc = 0.0;
  for (int ax = 0; ax < d; ++ax) {
    const int64_t st = ax == 0 ? 1 : (ax == 1 ? (int64_t)n : (int64_t)n * n);
    for (int sd = 0; sd < 2; ++sd) {
      const int s = sd ? 1 : -1;
      const int fit = P.aff_fit[t * 2 * d + 2 * ax + sd];
      const int js = P.aff_j[t * 2 * d + 2 * ax + sd];
      if (fit == -1 || fit >= P.nfit_cap) continue;
      if (fit >= 0) {
        for (int j = js; j <= W; ++j) {
          int pos = m[ax] + j * s;
          if (pos >= 0 && pos < n && P.phase[i + j * s * st] == ph) continue;   // back in phase: uses u
          acc = fma(P.a[W + j * s], P.G[(size_t)fit * W + (j - js)], acc);
        }
      } else {
        // outer box: ghosts from the degree-q line polynomial through the face value and
        // the nodes 2..q+1 counted from the face
        double face = 0.0;
        if (P.with_data) {
          int64_t off = 0, mul = 1;
          for (int k = 0; k < d; ++k) {
            if (k == ax) continue;
            off += m[k] * mul;
            mul *= n;
          }
          off += (int64_t)(2 * ax + sd) * mul;
          face = P.box[off];
        }
        for (int j = js; j <= W; ++j) {
          const int k = j - js;                  // ghost k+1 beyond the face
          double v = P.box_w[k][0] * face;
          for (int mm = 2; mm <= P.q + 1; ++mm) {
            int pos = s > 0 ? n - mm : mm - 1;
            v = fma(P.box_w[k][mm - 1], u[i + (int64_t)(pos - m[ax]) * st], v);
          }
          acc = fma(P.a[W + j * s], v, acc);
        }
      }
    }
  }
  w[i] += P.scale[ph ? 1 : 0] * acc;
}

__global__ void __launch_bounds__(256) k_ho_correct(CorrectParams P, const double* __restrict__ u,
                                                    double* __restrict__ w) {
  ho_correct_body(P, u, w, blockIdx.x * blockDim.x + threadIdx.x);
}

static StencilCoef stencil_coef(const Problem& P) {
  StencilCoef C;
  const double h2 = P.g.h * P.g.h;
  const double beta[2] = {P.desc.beta_minus, P.desc.beta_plus};
  for (int s = 0; s < 2; ++s) {
    C.c0[s] = P.g.dim * P.a[P.w] * beta[s] / h2;
    for (int j = 1; j <= kMaxW; ++j) C.cj[s][j - 1] = j <= P.w ? P.a[P.w + j] * beta[s] / h2 : 0.0;
  }
  return C;
}

void ho_stencil(Problem& P, const double* u, double* w, cudaStream_t s) {
  const GridView& g = P.g;
  const int T = 256;
  const int iface = P.desc.bc == IIM_BC_INTERFACE;
  StencilCoef C = stencil_coef(P);
  int grid = ceil_div(g.N, T);
  if (g.dim == 2) {
    if (P.w == 2) IIM_LAUNCH((k_ho_stencil<2, 2>), grid, T, 0, s, g, C, iface, u, P.phase, w);
    else IIM_LAUNCH((k_ho_stencil<2, 3>), grid, T, 0, s, g, C, iface, u, P.phase, w);
  } else {
    if (P.w == 2) IIM_LAUNCH((k_ho_stencil<3, 2>), grid, T, 0, s, g, C, iface, u, P.phase, w);
    else IIM_LAUNCH((k_ho_stencil<3, 3>), grid, T, 0, s, g, C, iface, u, P.phase, w);
  }
}

void ho_ghost(Problem& P, const double* u, bool with_data, cudaStream_t s) {
  const int T = 256;
  const int iface = P.desc.bc == IIM_BC_INTERFACE;
  GhostParams GP;
  GP.nfit = P.nfit_cap;
  GP.w = P.w;
  GP.rcap = P.rcap;
  GP.bc = P.desc.bc;
  GP.interface_ = iface;
  GP.with_data = with_data;
  GP.beta_p = P.desc.beta_plus;
  GP.beta_m = P.desc.beta_minus;
  GP.K = P.d_counts + 0;
  GP.fit_R = P.fit_R;
  GP.fit_nodes = P.fit_nodes;
  GP.fit_coef = P.fit_coef;
  GP.fit_cdat = P.fit_cdat;
  GP.g = P.d_g;
  GP.j0 = P.d_j0;
  GP.j1 = P.d_j1;
  GP.G = P.G;
  if (P.K_cap > 0) {
    // small blocks: a few thousand control points must still spread over all 152 SMs
    const int grid = ceil_div((int64_t)P.K_cap * kGhostLanes, 64);
    if (P.w == 2) IIM_LAUNCH(k_ho_ghost<2>, grid, 64, 0, s, GP, u);
    else IIM_LAUNCH(k_ho_ghost<3>, grid, 64, 0, s, GP, u);
  }
}

void ho_correct(Problem& P, const double* u, double* w, bool with_data, cudaStream_t s) {
  const GridView& g = P.g;
  const int T = 256;
  CorrectParams CP;
  CP.g = g;
  CP.w = P.w;
  CP.q = P.q;
  CP.with_data = with_data;
  CP.n_aff_cap = P.aff_cap;
  CP.nfit_cap = P.nfit_cap;
  CP.n_aff = P.d_counts + 1;
  CP.aff_node = P.aff_node;
  CP.aff_fit = P.aff_fit;
  CP.aff_j = P.aff_j;
  CP.G = P.G;
  CP.phase = P.phase;
  CP.box = P.d_box;
  for (int k = 0; k < 2 * kMaxW + 1; ++k) CP.a[k] = k < 2 * P.w + 1 ? P.a[k] : 0.0;
  const double h2 = g.h * g.h;
  CP.scale[0] = P.desc.beta_minus / h2;
  CP.scale[1] = P.desc.beta_plus / h2;
  for (int k = 0; k < kMaxW; ++k)
    for (int mm = 0; mm < 8; ++mm) CP.box_w[k][mm] = P.box_w[k][mm];
  if (P.aff_cap > 0) IIM_LAUNCH(k_ho_correct, ceil_div(P.aff_cap, 64), 64, 0, s, CP, u, w);
}

void ho_apply(Problem& P, const double* u, double* w, bool with_data, cudaStream_t s) {
  if (P.side && P.ev_fork && P.ev_join) {
    // the ghost values read only u: they are computed on the side stream beside the
    // stencil, and the corrections wait for both
    cudaEventRecord(P.ev_fork, s);
    cudaStreamWaitEvent(P.side, P.ev_fork, 0);
    ho_ghost(P, u, with_data, P.side);
    cudaEventRecord(P.ev_join, P.side);
    ho_stencil(P, u, w, s);
    cudaStreamWaitEvent(s, P.ev_join, 0);
  } else {
    ho_stencil(P, u, w, s);
    ho_ghost(P, u, with_data, s);
  }
  ho_correct(P, u, w, with_data, s);
}

__global__ void k_rhs_finish(GridView g, int interface_, const uint8_t* __restrict__ phase,
                             const double* __restrict__ f, const double* __restrict__ lg, double* __restrict__ b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  b[i] = (interface_ || phase[i]) ? f[i] - lg[i] : 0.0;
}

// b = f - L_Gamma u_Gamma: the operator applied to u = 0 with the data switched on
void compute_rhs(Problem& P, const double* f, cudaStream_t s) {
  double* zero = P.Z;                  // Z[0] is zeroed first: the apply reads it as u
  double* lg = P.tmp;
  cudaMemsetAsync(zero, 0, sizeof(double) * P.g.N, s);
  ho_apply(P, zero, lg, true, s);
  IIM_LAUNCH(k_rhs_finish, ceil_div(P.g.N, 256), 256, 0, s, P.g, P.desc.bc == IIM_BC_INTERFACE, P.phase, f, lg, P.b);
}


// ---------------------------------------------------------------------------- no-allocation apply
// The same three kernels as ho_apply, but the ghost values go to a file-scope
// device array instead of the problem's workspace.  kNoAllocGhostMax doubles
// (2 MiB) are reserved on every device that loads the library, for the life of
// the process.  All calls share the array, so calls that overlap on the device
// (other streams, other threads, other problems) race on it.  Each call writes
// every ghost value before it reads it, so nothing in the array has to be cleared.
namespace {
constexpr int64_t kNoAllocGhostMax = 1 << 18;
__device__ __align__(256) double g_noalloc_ghost[kNoAllocGhostMax];
constexpr int kNoAllocMaxDevices = 64;
double* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;
}  // namespace

iim_status ho_apply_noalloc(Problem& P, const double* u, double* w, bool with_data, cudaStream_t s) {
  const int64_t need = (int64_t)P.nfit_cap * P.w;
  if (need > kNoAllocGhostMax) {
    set_error("iim_apply_noalloc: the problem needs " + std::to_string(need) + " ghost values, more than the " +
              std::to_string(kNoAllocGhostMax) + " the static scratch holds");
    return IIM_ERR_CAPACITY;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    cudaGetLastError();
    set_error("iim_apply_noalloc: no usable current device");
    return IIM_ERR_CUDA;
  }
  double* G = nullptr;
  {
    // first call on this device: look up the device address of the array (the host
    // symbol is only a stand-in), with this device current
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_ghost);
      if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("iim_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return IIM_ERR_CUDA;
      }
      g_noalloc_addr[dev] = (double*)ptr;
    }
    G = g_noalloc_addr[dev];
  }
  ho_stencil(P, u, w, s);
  const int iface = P.desc.bc == IIM_BC_INTERFACE;
  GhostParams GP;
  GP.nfit = P.nfit_cap;
  GP.w = P.w;
  GP.rcap = P.rcap;
  GP.bc = P.desc.bc;
  GP.interface_ = iface;
  GP.with_data = with_data;
  GP.beta_p = P.desc.beta_plus;
  GP.beta_m = P.desc.beta_minus;
  GP.K = P.d_counts + 0;
  GP.fit_R = P.fit_R;
  GP.fit_nodes = P.fit_nodes;
  GP.fit_coef = P.fit_coef;
  GP.fit_cdat = P.fit_cdat;
  GP.g = P.d_g;
  GP.j0 = P.d_j0;
  GP.j1 = P.d_j1;
  GP.G = G;
  if (P.K_cap > 0) {
    const int grid = ceil_div((int64_t)P.K_cap * kGhostLanes, 64);
    if (P.w == 2) IIM_LAUNCH(k_ho_ghost<2>, grid, 64, 0, s, GP, u);
    else IIM_LAUNCH(k_ho_ghost<3>, grid, 64, 0, s, GP, u);
  }
  CorrectParams CP;
  const GridView& g = P.g;
  CP.g = g;
  CP.w = P.w;
  CP.q = P.q;
  CP.with_data = with_data;
  CP.n_aff_cap = P.aff_cap;
  CP.nfit_cap = P.nfit_cap;
  CP.n_aff = P.d_counts + 1;
  CP.aff_node = P.aff_node;
  CP.aff_fit = P.aff_fit;
  CP.aff_j = P.aff_j;
  CP.G = G;
  CP.phase = P.phase;
  CP.box = P.d_box;
  for (int k = 0; k < 2 * kMaxW + 1; ++k) CP.a[k] = k < 2 * P.w + 1 ? P.a[k] : 0.0;
  const double h2 = g.h * g.h;
  CP.scale[0] = P.desc.beta_minus / h2;
  CP.scale[1] = P.desc.beta_plus / h2;
  for (int k = 0; k < kMaxW; ++k)
    for (int mm = 0; mm < 8; ++mm) CP.box_w[k][mm] = P.box_w[k][mm];
  if (P.aff_cap > 0) IIM_LAUNCH(k_ho_correct, ceil_div(P.aff_cap, 64), 64, 0, s, CP, u, w);
  return IIM_OK;
}


// ---------------------------------------------------------------------------- batched engine
// Grouped forms of the three operator kernels.  A stencil item is four blocks of
// the single-problem launch; ghost and correction items are one block each.
template <int D, int W>
__global__ void __launch_bounds__(kEngThreads) k_eng_stencil(EngArgs A) {
  eng_for_items(A, kListStencil + (D - 2) * 2 + (W - 2), [&](int si, int item) {
    const SlotDev& s = A.slots[si];
    if (s.role == kRoleIdle) return;
    const double* u;
    double* w;
    eng_apply_io(s, u, w);
    const int64_t base = (int64_t)item * (4 * kEngThreads) + threadIdx.x;
    const int64_t N = s.g.N;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = base + k * kEngThreads;
      if (i < N) ho_stencil_node<D, W>(s.g, s.C, s.iface, u, s.phase, w, i);
    }
  });
}

template <int W>
__global__ void __launch_bounds__(64) k_eng_ghost(EngArgs A) {
  eng_for_items(A, kListGhost + (W - 2), [&](int si, int item) {
    const SlotDev& s = A.slots[si];
    if (s.role == kRoleIdle) return;
    const double* u;
    double* w;
    eng_apply_io(s, u, w);
    ho_ghost_body<W>(s.GP, u, item * 64 + threadIdx.x);
  });
}

__global__ void __launch_bounds__(64) k_eng_correct(EngArgs A) {
  eng_for_items(A, kListCorrect, [&](int si, int item) {
    const SlotDev& s = A.slots[si];
    if (s.role == kRoleIdle) return;
    const double* u;
    double* w;
    eng_apply_io(s, u, w);
    ho_correct_body(s.CP, u, w, item * 64 + threadIdx.x);
  });
}

void eng_launch_apply(const EngArgs& A, const unsigned char* present, cudaStream_t s) {
#define IIM_ENG_ST(D, W)                                                                                       \
  if (present[kListStencil + (D - 2) * 2 + (W - 2)])                                                          \
    IIM_LAUNCH((k_eng_stencil<D, W>), eng_grid((const void*)k_eng_stencil<D, W>, kEngThreads, 0), kEngThreads, 0, s, A);
  IIM_ENG_ST(2, 2) IIM_ENG_ST(2, 3) IIM_ENG_ST(3, 2) IIM_ENG_ST(3, 3)
#undef IIM_ENG_ST
  if (present[kListGhost + 0]) IIM_LAUNCH(k_eng_ghost<2>, eng_grid((const void*)k_eng_ghost<2>, 64, 0), 64, 0, s, A);
  if (present[kListGhost + 1]) IIM_LAUNCH(k_eng_ghost<3>, eng_grid((const void*)k_eng_ghost<3>, 64, 0), 64, 0, s, A);
  if (present[kListCorrect]) IIM_LAUNCH(k_eng_correct, eng_grid((const void*)k_eng_correct, 64, 0), 64, 0, s, A);
}

// the operator's per-problem parameters (homogeneous: the data enter through b)
void eng_operator_params(Problem& P, StencilCoef* C, GhostParams* GP, CorrectParams* CP) {
  *C = stencil_coef(P);
  GhostParams& G = *GP;
  G.nfit = P.nfit_cap;
  G.w = P.w;
  G.rcap = P.rcap;
  G.bc = P.desc.bc;
  G.interface_ = P.desc.bc == IIM_BC_INTERFACE;
  G.with_data = 0;
  G.beta_p = P.desc.beta_plus;
  G.beta_m = P.desc.beta_minus;
  G.K = P.d_counts + 0;
  G.fit_R = P.fit_R;
  G.fit_nodes = P.fit_nodes;
  G.fit_coef = P.fit_coef;
  G.fit_cdat = P.fit_cdat;
  G.g = P.d_g;
  G.j0 = P.d_j0;
  G.j1 = P.d_j1;
  G.G = P.G;
  CorrectParams& Q = *CP;
  Q.g = P.g;
  Q.w = P.w;
  Q.q = P.q;
  Q.with_data = 0;
  Q.n_aff_cap = P.aff_cap;
  Q.nfit_cap = P.nfit_cap;
  Q.n_aff = P.d_counts + 1;
  Q.aff_node = P.aff_node;
  Q.aff_fit = P.aff_fit;
  Q.aff_j = P.aff_j;
  Q.G = P.G;
  Q.phase = P.phase;
  Q.box = P.d_box;
  for (int k = 0; k < 2 * kMaxW + 1; ++k) Q.a[k] = k < 2 * P.w + 1 ? P.a[k] : 0.0;
  const double h2 = P.g.h * P.g.h;
  Q.scale[0] = P.desc.beta_minus / h2;
  Q.scale[1] = P.desc.beta_plus / h2;
  for (int k = 0; k < kMaxW; ++k)
    for (int mm = 0; mm < 8; ++mm) Q.box_w[k][mm] = P.box_w[k][mm];
}


// ---------------------------------------------------------------------------- boundary quantities, gradient
// Sec. 2.4: the boundary quantity the data do not prescribe, from row w of each fit:
// Dirichlet -> n . grad u(x_c) (derivative row, n out of Omega+), Neumann -> u(x_c)
// (Eq. 6, stored as coefficients over X_c plus 1/D_c times qbar).  Eight lanes per
// control point.
__global__ void __launch_bounds__(64) k_boundary_values(GhostParams P, const double* __restrict__ u,
                                                        double* __restrict__ out) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = gid / kGhostLanes, q = gid % kGhostLanes;
  const int K = *P.K;
  const bool live = c < K;
  double acc = 0.0;
  if (live) {
    const int R = P.fit_R[c];
    const int32_t* nodes = P.fit_nodes + (size_t)c * P.rcap;
    const double* row = P.fit_coef + ((size_t)c * (P.w + 1) + P.w) * P.rcap;
    for (int a = q; a < R; a += kGhostLanes) acc = fma(row[a], u[nodes[a]], acc);
  }
  acc = quad_sum(acc);
  if (live && q == 0) out[c] = acc + P.fit_cdat[(size_t)c * (P.w + 1) + P.w] * P.g[c];
}

// centred first-derivative stencil b_{-w..w} of order 2w (odd, b_0 = 0): the unique
// stencil exact for polynomials of degree <= 2w (2/3, -1/12 for w = 2; 3/4, -3/20,
// 1/60 for w = 3)
struct GradCoef {
  double b[2 * kMaxW + 1];
};

static GradCoef grad_coef(int w) {
  GradCoef B;
  const double h2[2] = {2.0 / 3.0, -1.0 / 12.0};
  const double h3[3] = {3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0};
  for (int k = 0; k < 2 * kMaxW + 1; ++k) B.b[k] = 0.0;
  for (int j = 1; j <= w; ++j) {
    const double v = w == 2 ? h2[j - 1] : h3[j - 1];
    B.b[w + j] = v;
    B.b[w - j] = -v;
  }
  return B;
}

// grad u by the centred first-derivative stencil b of the scheme's order: neighbours
// out of phase (or outside the box) contribute nothing here; their ghost values are
// added by k_grad_correct.  out is [dim][N]; zero at nodes that are not unknowns.
template <int D, int W>
__global__ void __launch_bounds__(256) k_grad_stencil(GridView g, GradCoef B, int interface_,
                                                      const double* __restrict__ u,
                                                      const uint8_t* __restrict__ phase, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  const int n = g.n;
  const uint8_t ph = phase[i];
  if (!interface_ && !ph) {
#pragma unroll
    for (int ax = 0; ax < D; ++ax) out[(size_t)ax * g.N + i] = 0.0;
    return;
  }
  int m[3];
  m[0] = (int)(i % n);
  const int64_t r = i / n;
  m[1] = (int)(r % n);
  m[2] = D > 2 ? (int)(r / n) : 0;
  const double ih = 1.0 / g.h;
#pragma unroll
  for (int ax = 0; ax < D; ++ax) {
    const int64_t st = ax == 0 ? 1 : (ax == 1 ? (int64_t)n : (int64_t)n * n);
    double acc = 0.0;
#pragma unroll
    for (int j = 1; j <= W; ++j) {
      double lv = 0.0, rv = 0.0;
      if (m[ax] - j >= 0 && phase[i - j * st] == ph) lv = u[i - j * st];
      if (m[ax] + j < n && phase[i + j * st] == ph) rv = u[i + j * st];
      acc = fma(B.b[W + j], rv - lv, acc);
    }
    out[(size_t)ax * g.N + i] = acc * ih;
  }
}

// ghost contributions to the gradient at the affected nodes (the walk rules of k_ho_correct)
__global__ void __launch_bounds__(64) k_grad_correct(CorrectParams P, GradCoef B,
                                                     const double* __restrict__ u, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *P.n_aff || t >= P.n_aff_cap) return;
  const GridView& g = P.g;
  const int n = g.n, d = g.dim, W = P.w;
  const int64_t i = P.aff_node[t];
  int m[3];
  m[0] = (int)(i % n);
  const int64_t r = i / n;
  m[1] = (int)(r % n);
  m[2] = d > 2 ? (int)(r / n) : 0;
  const uint8_t ph = P.phase[i];
  const double ih = 1.0 / g.h;
  for (int ax = 0; ax < d; ++ax) {
    const int64_t st = ax == 0 ? 1 : (ax == 1 ? (int64_t)n : (int64_t)n * n);
    double acc = 0.0;
    for (int sd = 0; sd < 2; ++sd) {
      const int s = sd ? 1 : -1;
      const int fit = P.aff_fit[t * 2 * d + 2 * ax + sd];
      const int js = P.aff_j[t * 2 * d + 2 * ax + sd];
      if (fit == -1 || fit >= P.nfit_cap) continue;
      if (fit >= 0) {
        for (int j = js; j <= W; ++j) {
          const int pos = m[ax] + j * s;
          if (pos >= 0 && pos < n && P.phase[i + j * s * st] == ph) continue;
          acc = fma(B.b[W + j * s], P.G[(size_t)fit * W + (j - js)], acc);
        }
      } else {
        double face = 0.0;
        if (P.with_data) {
          int64_t off = 0, mul = 1;
          for (int k = 0; k < d; ++k) {
            if (k == ax) continue;
            off += m[k] * mul;
            mul *= n;
          }
          off += (int64_t)(2 * ax + sd) * mul;
          face = P.box[off];
        }
        for (int j = js; j <= W; ++j) {
          const int k = j - js;
          double v = P.box_w[k][0] * face;
          for (int mm = 2; mm <= P.q + 1; ++mm) {
            const int pos = s > 0 ? n - mm : mm - 1;
            v = fma(P.box_w[k][mm - 1], u[i + (int64_t)(pos - m[ax]) * st], v);
          }
          acc = fma(B.b[W + j * s], v, acc);
        }
      }
    }
    out[(size_t)ax * g.N + i] += acc * ih;
  }
}

iim_status boundary_values(Problem& P, const double* u, double* out, cudaStream_t s) {
  if (P.desc.bc == IIM_BC_INTERFACE) {
    set_error("boundary values are defined for boundary problems");
    return IIM_ERR_INVALID_ARG;
  }
  StencilCoef C;
  GhostParams GP;
  CorrectParams CP;
  eng_operator_params(P, &C, &GP, &CP);
  if (P.K_cap > 0)
    IIM_LAUNCH(k_boundary_values, ceil_div((int64_t)P.K_cap * kGhostLanes, 64), 64, 0, s, GP, u, out);
  return IIM_OK;
}

iim_status gradient(Problem& P, const double* u, double* grad, cudaStream_t s) {
  const GridView& g = P.g;
  const GradCoef b_dev = grad_coef(P.w);
  const int iface = P.desc.bc == IIM_BC_INTERFACE;
  const int grid = ceil_div(g.N, 256);
  if (g.dim == 2) {
    if (P.w == 2) IIM_LAUNCH((k_grad_stencil<2, 2>), grid, 256, 0, s, g, b_dev, iface, u, P.phase, grad);
    else IIM_LAUNCH((k_grad_stencil<2, 3>), grid, 256, 0, s, g, b_dev, iface, u, P.phase, grad);
  } else {
    if (P.w == 2) IIM_LAUNCH((k_grad_stencil<3, 2>), grid, 256, 0, s, g, b_dev, iface, u, P.phase, grad);
    else IIM_LAUNCH((k_grad_stencil<3, 3>), grid, 256, 0, s, g, b_dev, iface, u, P.phase, grad);
  }
  ho_ghost(P, u, true, s);                        // ghost values with the problem's data
  StencilCoef C;
  GhostParams GP;
  CorrectParams CP;
  eng_operator_params(P, &C, &GP, &CP);
  CP.with_data = 1;
  if (P.aff_cap > 0) IIM_LAUNCH(k_grad_correct, ceil_div(P.aff_cap, 64), 64, 0, s, CP, b_dev, u, grad);
  return IIM_OK;
}

}  // namespace iim
