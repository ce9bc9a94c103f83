// Shortley-Weller geometric multigrid V-cycle (paper Sec. 3.3), FP32 or FP64.
//
// Cell-centred levels n, n/2, ...; red-black Gauss-Seidel (red = even index
// sum, red first); residual + restriction as the mean of the 2^d children with
// zeros outside the domain; bi/trilinear interpolation with zeros outside the
// domain (Dirichlet, interface) or the mean of the in-domain coarse neighbours
// (Neumann, Sec. 3.3); a dense direct solve on the coarsest level.  Interface
// problems run on lap(u) = f/beta per phase (Sec. 3.3): the FP64 Krylov vector
// is divided by beta_sigma when it enters the FP32 hierarchy.
#include "kernels.cuh"

namespace iim {

template <typename T>
struct LevelView {
  GridView g;
  const int32_t* aux;
  const T* tab;
};

template <typename T>
__device__ inline T tabv(const LevelView<T>& L, int r, int k) {
  return L.tab[(size_t)r * (2 * L.g.dim + 1) + k];
}

__device__ inline void idx3(const GridView& g, int64_t i, int* m) {
  m[0] = (int)(i % g.n);
  int64_t r = i / g.n;
  m[1] = (int)(r % g.n);
  m[2] = g.dim > 2 ? (int)(r / g.n) : 0;
}

// (L u)_i without the diagonal term: sum of off-diagonal coefficients times neighbours
template <typename T>
__device__ inline T offdiag_sum(const LevelView<T>& L, int64_t i, const int* m, int a, const T* __restrict__ u) {
  const GridView& g = L.g;
  T s = 0;
  if (a == -1) {
    const T ih2 = (T)(1.0 / (g.h * g.h));
    for (int ax = 0; ax < g.dim; ++ax) {
      int64_t st = ax == 0 ? 1 : (ax == 1 ? (int64_t)g.n : (int64_t)g.n * g.n);
      s += u[i - st] + u[i + st];
    }
    return s * ih2;
  }
  for (int ax = 0; ax < g.dim; ++ax) {
    int64_t st = ax == 0 ? 1 : (ax == 1 ? (int64_t)g.n : (int64_t)g.n * g.n);
    T cl = tabv(L, a, 1 + 2 * ax), cr = tabv(L, a, 2 + 2 * ax);
    if (cl != (T)0 && m[ax] > 0) s += cl * u[i - st];
    if (cr != (T)0 && m[ax] < g.n - 1) s += cr * u[i + st];
  }
  return s;
}

template <typename T>
__device__ inline T diag_of(const LevelView<T>& L, int a) {
  if (a == -1) return (T)(-2.0 * L.g.dim / (L.g.h * L.g.h));
  return tabv(L, a, 0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_smooth(LevelView<T> L, T* __restrict__ u, const T* __restrict__ f,
                                                int colour) {
  // one thread per node of the colour: node = 2 * t + parity fix-up along x
  const GridView& g = L.g;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t rows = g.N / g.n;
  int64_t half = (g.n + 1) / 2;
  if (t >= rows * half) return;
  int64_t row = t / half;
  int xi = (int)(t - row * half) * 2;
  int ry = (int)(row % g.n), rz = g.dim > 2 ? (int)(row / g.n) : 0;
  if (((xi + ry + rz) & 1) != colour) xi += 1;
  if (xi >= g.n) return;
  int64_t i = row * g.n + xi;
  int a = L.aux[i];
  if (a == -2) return;
  int m[3] = {xi, ry, rz};
  T dg = diag_of(L, a);
  T s = offdiag_sum(L, i, m, a, u);
  u[i] = dg != (T)0 ? (f[i] - s) / dg : (T)0;
}

// coarse f = mean over the 2^d children of r = f - L u (zero at non-unknowns)
template <typename T>
__global__ void __launch_bounds__(256) k_resid_restrict(LevelView<T> F, const T* __restrict__ u,
                                                        const T* __restrict__ f, GridView gc,
                                                        const int32_t* __restrict__ aux_c, T* __restrict__ fc) {
  int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= gc.N) return;
  if (aux_c[I] == -2) { fc[I] = (T)0; return; }
  int mc[3];
  idx3(gc, I, mc);
  const GridView& g = F.g;
  T acc = 0;
  const int nch = 1 << g.dim;
  for (int c = 0; c < nch; ++c) {
    int m[3] = {2 * mc[0] + (c & 1), 2 * mc[1] + ((c >> 1) & 1), g.dim > 2 ? 2 * mc[2] + ((c >> 2) & 1) : 0};
    int64_t i = m[0] + (int64_t)g.n * m[1] + (int64_t)g.n * g.n * m[2];
    int a = F.aux[i];
    if (a == -2) continue;
    T r = f[i] - (diag_of(F, a) * u[i] + offdiag_sum(F, i, m, a, u));
    acc += r;
  }
  fc[I] = acc / (T)nch;
}

// u_fine += P e_coarse at fine unknowns
template <typename T>
__global__ void __launch_bounds__(256) k_prolong(GridView gf, const int32_t* __restrict__ aux_f, T* __restrict__ uf,
                                                 GridView gc, const int32_t* __restrict__ aux_c,
                                                 const T* __restrict__ ec, int neumann) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= gf.N) return;
  if (aux_f[i] == -2) return;
  int m[3];
  idx3(gf, i, m);
  int I[3] = {m[0] >> 1, m[1] >> 1, m[2] >> 1};
  int sg[3] = {(m[0] & 1) ? 1 : -1, (m[1] & 1) ? 1 : -1, (m[2] & 1) ? 1 : -1};
  T acc = 0;
  int cnt = 0;
  const int nsel = 1 << gf.dim;
  for (int sel = 0; sel < nsel; ++sel) {
    int c[3];
    T wgt = 1;
    bool inb = true;
    for (int k = 0; k < 3; ++k) {
      int b = (sel >> k) & 1;
      c[k] = k < gf.dim ? I[k] + b * sg[k] : 0;
      if (k < gf.dim) {
        if (c[k] < 0 || c[k] >= gc.n) inb = false;
        wgt *= b ? (T)0.25 : (T)0.75;
      }
    }
    if (!inb) continue;
    int64_t ci = c[0] + (int64_t)gc.n * c[1] + (int64_t)gc.n * gc.n * c[2];
    if (aux_c[ci] == -2) continue;
    if (neumann) { acc += ec[ci]; ++cnt; }
    else acc += wgt * ec[ci];
  }
  if (neumann) acc = cnt > 0 ? acc / (T)cnt : (T)0;
  uf[i] += acc;
}

// f_fine = v * scale / beta_sigma at unknowns (FP64 -> level precision)
template <typename T>
__global__ void k_bridge_in(GridView g, const double* __restrict__ v, const double* __restrict__ scale,
                            const uint8_t* __restrict__ phase, const int32_t* __restrict__ aux, double inv_bp,
                            double inv_bm, T* __restrict__ f) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  if (aux[i] == -2) { f[i] = (T)0; return; }
  const T sc = (T)((scale ? *scale : 1.0) * (phase[i] ? inv_bp : inv_bm));
  f[i] = (T)v[i] * sc;
}

template <typename T>
__global__ void k_zero(T* __restrict__ u, int64_t N) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) u[i] = (T)0;
}

template <typename T>
__global__ void k_bridge_out(GridView g, const T* __restrict__ u, double* __restrict__ z) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  z[i] = (double)u[i];
}

// ---------------------------------------------------------------------------- coarsest level
// dense coarse matrix (row major, nu x nu) from the level's stencil
template <typename T>
__global__ void k_coarse_assemble(LevelView<double> L, const int32_t* __restrict__ map, int nu,
                                  const int32_t* __restrict__ inv, T* __restrict__ A) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nu) return;
  for (int c = 0; c < nu; ++c) A[(size_t)r * nu + c] = 0;
  int64_t i = map[r];
  int a = L.aux[i];
  int m[3];
  idx3(L.g, i, m);
  A[(size_t)r * nu + r] = (T)diag_of(L, a);
  const GridView& g = L.g;
  for (int ax = 0; ax < g.dim; ++ax) {
    int64_t st = ax == 0 ? 1 : (ax == 1 ? (int64_t)g.n : (int64_t)g.n * g.n);
    for (int s = -1; s <= 1; s += 2) {
      int pos = m[ax] + s;
      if (pos < 0 || pos >= g.n) continue;
      double cf = a == -1 ? 1.0 / (g.h * g.h) : tabv(L, a, (s < 0 ? 1 : 2) + 2 * ax);
      if (cf == 0.0) continue;
      int col = inv[i + s * st];
      if (col >= 0) A[(size_t)r * nu + col] = (T)cf;
    }
  }
}

__global__ void k_coarse_map(GridView g, const int32_t* __restrict__ aux, const int32_t* __restrict__ idx,
                             int32_t* __restrict__ map, int32_t* __restrict__ inv) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  if (aux[i] == -2) { inv[i] = -1; return; }
  int k = idx[i];
  map[k] = (int32_t)i;
  inv[i] = k;
}

__global__ void k_unknown_flag(GridView g, const int32_t* __restrict__ aux, int32_t* __restrict__ flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < g.N) flag[i] = aux[i] != -2;
}

// LU with partial pivoting (one CTA), then the explicit inverse (column by column)
template <typename T>
__global__ void k_coarse_lu(T* __restrict__ A, int nu, int32_t* __restrict__ piv, T* __restrict__ inv,
                            int* status) {
  __shared__ int s_p;
  __shared__ T s_best[32];
  __shared__ int s_bi[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k < nu; ++k) {
    // pivot search
    T best = -1;
    int bi = k;
    for (int r = k + tid; r < nu; r += nt) {
      T v = fabs(A[(size_t)r * nu + k]);
      if (v > best) { best = v; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((tid & 31) == 0) { s_best[tid >> 5] = best; s_bi[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      T b0 = s_best[0];
      int i0 = s_bi[0];
      for (int w = 1; w < nt / 32; ++w)
        if (s_best[w] > b0 || (s_best[w] == b0 && s_bi[w] < i0)) { b0 = s_best[w]; i0 = s_bi[w]; }
      s_p = i0;
      piv[k] = i0;
      if (!(b0 > 0)) set_status(status, IIM_ERR_SINGULAR);
    }
    __syncthreads();
    int p = s_p;
    if (p != k)
      for (int c = tid; c < nu; c += nt) {
        T t = A[(size_t)k * nu + c];
        A[(size_t)k * nu + c] = A[(size_t)p * nu + c];
        A[(size_t)p * nu + c] = t;
      }
    __syncthreads();
    T d = A[(size_t)k * nu + k];
    for (int r = k + 1 + tid; r < nu; r += nt) A[(size_t)r * nu + k] /= d;
    __syncthreads();
    int rem = nu - k - 1;
    for (int e = tid; e < rem * rem; e += nt) {
      int r = k + 1 + e / rem, c = k + 1 + e % rem;
      A[(size_t)r * nu + c] -= A[(size_t)r * nu + k] * A[(size_t)k * nu + c];
    }
    __syncthreads();
  }
  // inverse: solve L U x = P e_j, one warp per column
  const int lane = tid & 31, wid = tid >> 5, nw = nt / 32;
  for (int j = wid; j < nu; j += nw) {
    T* x = inv + (size_t)j;      // column j of the inverse, stride nu (row major inverse)
    // b = P e_j : apply the row swaps to e_j
    for (int r = lane; r < nu; r += 32) x[(size_t)r * nu] = (r == j) ? (T)1 : (T)0;
    __syncwarp();
    if (lane == 0)
      for (int k = 0; k < nu; ++k) {
        int p = piv[k];
        if (p != k) { T t = x[(size_t)k * nu]; x[(size_t)k * nu] = x[(size_t)p * nu]; x[(size_t)p * nu] = t; }
      }
    __syncwarp();
    for (int r = 0; r < nu; ++r) {                 // forward, unit lower
      T part = 0;
      for (int c = lane; c < r; c += 32) part += A[(size_t)r * nu + c] * x[(size_t)c * nu];
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) x[(size_t)r * nu] -= part;
      __syncwarp();
    }
    for (int r = nu - 1; r >= 0; --r) {            // backward
      T part = 0;
      for (int c = r + 1 + lane; c < nu; c += 32) part += A[(size_t)r * nu + c] * x[(size_t)c * nu];
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) x[(size_t)r * nu] = (x[(size_t)r * nu] - part) / A[(size_t)r * nu + r];
      __syncwarp();
    }
  }
}

// u_c = A^-1 f_c on the coarsest level (one CTA)
template <typename T>
__global__ void k_coarse_solve(int nu, const int32_t* __restrict__ map, const T* __restrict__ inv,
                               const T* __restrict__ f, T* __restrict__ u, int64_t Nc) {
  extern __shared__ unsigned char smraw[];
  T* fb = (T*)smraw;
  for (int64_t i = threadIdx.x; i < Nc; i += blockDim.x) u[i] = (T)0;
  for (int r = threadIdx.x; r < nu; r += blockDim.x) fb[r] = f[map[r]];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x / 32;
  for (int r = wid; r < nu; r += nw) {
    T s = 0;
    for (int c = lane; c < nu; c += 32) s += inv[(size_t)r * nu + c] * fb[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) u[map[r]] = s;
  }
}

// ---------------------------------------------------------------------------- host side
template <typename T>
static LevelView<T> view(const Level& L) {
  LevelView<T> v;
  v.g = L.g;
  v.aux = L.aux;
  v.tab = (const T*)(sizeof(T) == 8 ? (const void*)L.tab64 : (const void*)L.tab32);
  return v;
}

template <typename T>
static void vcycle(Problem& P, size_t l, cudaStream_t s) {
  const int Tn = 256;
  Level& L = P.lv[l];
  T* u = (T*)L.u;
  T* f = (T*)L.f;
  if (l + 1 == P.lv.size()) {
    const T* inv = (const T*)(sizeof(T) == 8 ? (void*)P.coarse_lu64 : (void*)P.coarse_lu32);
    IIM_LAUNCH(k_coarse_solve<T>, 1, 1024, sizeof(T) * (P.coarse_nu + 1), s, P.coarse_nu, P.coarse_map,
               inv + (size_t)P.coarse_nu * P.coarse_nu, f, u, L.g.N);
    return;
  }
  LevelView<T> V = view<T>(L);
  const int64_t ncol = (L.g.N / L.g.n) * ((L.g.n + 1) / 2);
  IIM_LAUNCH(k_zero<T>, ceil_div(L.g.N, Tn), Tn, 0, s, u, L.g.N);
  for (int it = 0; it < P.opt.nu1; ++it)
    for (int c = 0; c < 2; ++c) IIM_LAUNCH(k_smooth<T>, ceil_div(ncol, Tn), Tn, 0, s, V, u, f, c);
  Level& C = P.lv[l + 1];
  IIM_LAUNCH(k_resid_restrict<T>, ceil_div(C.g.N, Tn), Tn, 0, s, V, u, f, C.g, C.aux, (T*)C.f);
  vcycle<T>(P, l + 1, s);
  IIM_LAUNCH(k_prolong<T>, ceil_div(L.g.N, Tn), Tn, 0, s, L.g, L.aux, u, C.g, C.aux, (const T*)C.u,
             P.desc.bc == IIM_BC_NEUMANN);
  for (int it = 0; it < P.opt.nu2; ++it)
    for (int c = 0; c < 2; ++c) IIM_LAUNCH(k_smooth<T>, ceil_div(ncol, Tn), Tn, 0, s, V, u, f, c);
}

template <typename T>
static void precondition_t(Problem& P, const double* v, const double* vscale, double* z, cudaStream_t s) {
  Level& L = P.lv[0];
  const int Tn = 256;
  IIM_LAUNCH(k_bridge_in<T>, ceil_div(L.g.N, Tn), Tn, 0, s, L.g, v, vscale, P.phase, L.aux,
             1.0 / P.desc.beta_plus, 1.0 / P.desc.beta_minus, (T*)L.f);
  vcycle<T>(P, 0, s);
  IIM_LAUNCH(k_bridge_out<T>, ceil_div(L.g.N, Tn), Tn, 0, s, L.g, (const T*)L.u, z);
}

void mg_precondition(Problem& P, const double* v, const double* vscale, double* z, cudaStream_t s) {
  if (P.opt.mg_precision == IIM_MG_FP64) precondition_t<double>(P, v, vscale, z, s);
  else precondition_t<float>(P, v, vscale, z, s);
}

// coarse matrix, LU and inverse; coarse_lu{64,32} hold [A (nu*nu) | inverse (nu*nu)]
void mg_coarse_factor(Problem& P, cudaStream_t s) {
  Level& C = P.lv.back();
  const int nu = P.coarse_nu;
  if (nu <= 0) return;
  const int Tn = 256;
  IIM_LAUNCH(k_unknown_flag, ceil_div(C.g.N, Tn), Tn, 0, s, C.g, C.aux, C.flag);
  scan_exclusive(C.flag, C.idx, C.g.N, P.d_counts + 7, P.scan_scratch, s);
  int32_t* inv = C.flag;            // reuse: node -> unknown index
  IIM_LAUNCH(k_coarse_map, ceil_div(C.g.N, Tn), Tn, 0, s, C.g, C.aux, C.idx, P.coarse_map, inv);
  LevelView<double> V = view<double>(C);
  if (P.opt.mg_precision == IIM_MG_FP64) {
    IIM_LAUNCH(k_coarse_assemble<double>, ceil_div(nu, 128), 128, 0, s, V, P.coarse_map, nu, inv, P.coarse_lu64);
    IIM_LAUNCH(k_coarse_lu<double>, 1, 1024, 0, s, P.coarse_lu64, nu, P.coarse_piv,
               P.coarse_lu64 + (size_t)nu * nu, P.d_status);
  } else {
    IIM_LAUNCH(k_coarse_assemble<float>, ceil_div(nu, 128), 128, 0, s, V, P.coarse_map, nu, inv, P.coarse_lu32);
    IIM_LAUNCH(k_coarse_lu<float>, 1, 1024, 0, s, P.coarse_lu32, nu, P.coarse_piv, P.coarse_lu32 + (size_t)nu * nu,
               P.d_status);
  }
}

}  // namespace iim
