// Shortley-Weller geometric multigrid V-cycle (paper Sec. 3.3), FP32 or FP64.
//
// Cell-centred levels n, n/2, ...; red-black Gauss-Seidel (red = even index
// sum, red first); residual + restriction as the mean of the 2^d children with
// zeros outside the domain; bi/trilinear interpolation with zeros outside the
// domain (Dirichlet, interface) or the mean of the in-domain coarse neighbours
// (Neumann, Sec. 3.3); a dense direct solve on the coarsest level.  Interface
// problems run on lap(u) = f/beta per phase (Sec. 3.3): the FP64 Krylov vector
// is divided by beta_sigma when it enters the FP32 hierarchy.
#include <algorithm>
#include <utility>

#include "engine.cuh"
#include "mg_rb.cuh"

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
__device__ inline T offdiag_sum(const LevelView<T>& L, T ih2, int64_t i, const int* m, int a, const T* __restrict__ u) {
  const GridView& g = L.g;
  T s = 0;
  if (a == -1) {
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
__device__ inline T diag_of(const LevelView<T>& L, T dreg, int a) {
  if (a == -1) return dreg;
  return tabv(L, a, 0);
}

template <typename T>
__device__ __forceinline__ void smooth_body(const LevelView<T>& L, T ih2, T dreg, T* __restrict__ u,
                                            const T* __restrict__ f, int f_bf16, int colour, int64_t t) {
  // one thread per node of the colour: node = 2 * t + parity fix-up along x
  const GridView& g = L.g;
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
  T dg = diag_of(L, dreg, a);
  T s = offdiag_sum(L, ih2, i, m, a, u);
  u[i] = dg != (T)0 ? (load_f(f, i, f_bf16) - s) / dg : (T)0;
}

template <typename T>
__global__ void __launch_bounds__(256) k_smooth(LevelView<T> L, T ih2, T dreg, T* __restrict__ u,
                                                const T* __restrict__ f, int f_bf16, int colour) {
  smooth_body<T>(L, ih2, dreg, u, f, f_bf16, colour, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// coarse f = mean over the 2^d children of r = f - L u (zero at non-unknowns)
template <typename T>
__device__ __forceinline__ void resid_restrict_body(const LevelView<T>& F, T ih2, T dreg, const T* __restrict__ u,
                                                    const T* __restrict__ f, int f_in_bf16, const GridView& gc,
                                                    const int32_t* __restrict__ aux_c, T* __restrict__ fc, int64_t I,
                                                    int f_bf16) {
  if (I >= gc.N) return;
  if (aux_c[I] == -2) { store_f(fc, I, (T)0, f_bf16); return; }
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
    T r = load_f(f, i, f_in_bf16) - (diag_of(F, dreg, a) * u[i] + offdiag_sum(F, ih2, i, m, a, u));
    acc += r;
  }
  store_f(fc, I, acc / (T)nch, f_bf16);
}

template <typename T>
__global__ void __launch_bounds__(256) k_resid_restrict(LevelView<T> F, T ih2, T dreg, const T* __restrict__ u,
                                                        const T* __restrict__ f, int f_in_bf16, GridView gc,
                                                        const int32_t* __restrict__ aux_c, T* __restrict__ fc,
                                                        int f_bf16) {
  resid_restrict_body<T>(F, ih2, dreg, u, f, f_in_bf16, gc, aux_c, fc, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                         f_bf16);
}

// u_fine += P e_coarse at fine unknowns
template <typename T>
__device__ __forceinline__ void prolong_body(const GridView& gf, const int32_t* __restrict__ aux_f, T* __restrict__ uf,
                                             const GridView& gc, const int32_t* __restrict__ aux_c,
                                             const T* __restrict__ ec, int neumann, int64_t i) {
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

template <typename T>
__global__ void __launch_bounds__(256) k_prolong(GridView gf, const int32_t* __restrict__ aux_f, T* __restrict__ uf,
                                                 GridView gc, const int32_t* __restrict__ aux_c,
                                                 const T* __restrict__ ec, int neumann) {
  prolong_body<T>(gf, aux_f, uf, gc, aux_c, ec, neumann, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// f_fine = v * scale / beta_sigma at unknowns (FP64 -> level precision)
template <typename T>
__device__ __forceinline__ void bridge_in_body(const GridView& g, const double* __restrict__ v,
                                               const double* __restrict__ scale, const uint8_t* __restrict__ phase,
                                               const int32_t* __restrict__ aux, double inv_bp, double inv_bm,
                                               T* __restrict__ f, int64_t i) {
  if (i >= g.N) return;
  if (aux[i] == -2) { f[i] = (T)0; return; }
  const T sc = (T)((scale ? *scale : 1.0) * (phase[i] ? inv_bp : inv_bm));
  f[i] = (T)v[i] * sc;
}

template <typename T>
__global__ void k_bridge_in(GridView g, const double* __restrict__ v, const double* __restrict__ scale,
                            const uint8_t* __restrict__ phase, const int32_t* __restrict__ aux, double inv_bp,
                            double inv_bm, T* __restrict__ f) {
  bridge_in_body<T>(g, v, scale, phase, aux, inv_bp, inv_bm, f, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
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
__global__ void k_coarse_assemble(LevelView<double> L, const int32_t* __restrict__ map, const int* __restrict__ nu_dev,
                                  int ld, const int32_t* __restrict__ inv, T* __restrict__ A, int aug, int* status) {
  // The coarse system of the current set-up in the leading n x n block (n = nu + aug, nu the
  // coarsest level's unknowns, counted on the device) of an array of fixed stride ld (the
  // level's node count + aug), so that a later set-up with another geometry needs no other
  // size: rows r < nu the SW operator; augmented (pure Neumann, Sec. 2.3): a last column and
  // row of ones over the unknowns and a zero corner
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int nu = *nu_dev, n = nu + aug;
  if (nu < 0 || n > ld) {              // more unknowns than the system has room for
    if (r == 0) set_status(status, IIM_ERR_CAPACITY);
    return;
  }
  if (r >= n) return;
  for (int c = 0; c < n; ++c) A[(size_t)r * ld + c] = (aug && c == nu && r < nu) ? (T)1 : (T)0;
  if (r == nu) {                       // the augmentation row
    for (int c = 0; c < nu; ++c) A[(size_t)r * ld + c] = 1;
    return;
  }
  int64_t i = map[r];
  int a = L.aux[i];
  int m[3];
  idx3(L.g, i, m);
  A[(size_t)r * ld + r] = (T)diag_of(L, -2.0 * L.g.dim / (L.g.h * L.g.h), a);
  const GridView& g = L.g;
  for (int ax = 0; ax < g.dim; ++ax) {
    int64_t st = ax == 0 ? 1 : (ax == 1 ? (int64_t)g.n : (int64_t)g.n * g.n);
    for (int s = -1; s <= 1; s += 2) {
      int pos = m[ax] + s;
      if (pos < 0 || pos >= g.n) continue;
      double cf = a == -1 ? 1.0 / (g.h * g.h) : tabv(L, a, (s < 0 ? 1 : 2) + 2 * ax);
      if (cf == 0.0) continue;
      int col = inv[i + s * st];
      if (col >= 0) A[(size_t)r * ld + col] = (T)cf;
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

// LU with partial pivoting (one CTA), then the explicit inverse, of the leading n x n block
// (n read on the device) of the stride-ld array Ag; the inverse goes to inv with stride ld.
// With room for it (smem_elems elements of dynamic shared memory) the matrix, and then also
// the inverse, are worked on in shared memory (stride n).
template <typename T>
__global__ void k_coarse_lu(T* __restrict__ Ag, int ld, const int* __restrict__ nu_dev, int aug,
                            int32_t* __restrict__ piv, T* __restrict__ inv, int* status, size_t smem_elems) {
  extern __shared__ unsigned char smraw[];
  __shared__ int s_p;
  __shared__ T s_best[32];
  __shared__ int s_bi[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nu = *nu_dev + aug;           // the system's dimension (the name of the loops below)
  if (nu <= 0 || nu > ld) return;         // out of range: reported by k_coarse_assemble
  const size_t nn = (size_t)nu * nu;
  const int in_smem = 2 * nn <= smem_elems ? 2 : (nn <= smem_elems ? 1 : 0);
  const int la = in_smem ? nu : ld;       // stride of the working copy
  T* A = in_smem ? (T*)smraw : Ag;
  if (in_smem)
    for (size_t e = tid; e < nn; e += nt) A[e] = Ag[(e / nu) * ld + e % nu];
  __syncthreads();
  for (int k = 0; k < nu; ++k) {
    T best = -1;
    int bi = k;
    for (int r = k + tid; r < nu; r += nt) {
      T v = fabs(A[(size_t)r * la + k]);
      if (v > best) { best = v; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      T ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((tid & 31) == 0) { s_best[tid >> 5] = best; s_bi[tid >> 5] = bi; }
    __syncthreads();
    if (tid < 32) {                     // the warps' candidates, reduced by the first warp
      T b0 = tid < nt / 32 ? s_best[tid] : (T)-1;
      int i0 = tid < nt / 32 ? s_bi[tid] : nu;
      for (int o = 16; o > 0; o >>= 1) {
        T ob = __shfl_xor_sync(0xffffffffu, b0, o);
        int oi = __shfl_xor_sync(0xffffffffu, i0, o);
        if (ob > b0 || (ob == b0 && oi < i0)) { b0 = ob; i0 = oi; }
      }
      if (tid == 0) {
        s_p = i0;
        piv[k] = i0;
        if (!(b0 > 0)) set_status(status, IIM_ERR_SINGULAR);
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p != k)
      for (int c = tid; c < nu; c += nt) {
        T t = A[(size_t)k * la + c];
        A[(size_t)k * la + c] = A[(size_t)p * la + c];
        A[(size_t)p * la + c] = t;
      }
    __syncthreads();
    const T d = A[(size_t)k * la + k];
    const int rem = nu - k - 1;
    for (int r = k + 1 + tid; r < nu; r += nt) A[(size_t)r * la + k] /= d;
    __syncthreads();
    for (int e = tid; e < rem * rem; e += nt) {
      int r = k + 1 + e / rem, c = k + 1 + e % rem;
      A[(size_t)r * la + c] -= A[(size_t)r * la + k] * A[(size_t)k * la + c];
    }
    __syncthreads();
  }
  if (in_smem)
    for (size_t e = tid; e < nn; e += nt) Ag[(e / nu) * ld + e % nu] = A[e];
  __syncthreads();
  if (in_smem == 2) {
    // inverse in shared memory: X = U^-1 L^-1 P, all columns at once, one row per step.
    // Column j is handled by G consecutive lanes that split the row's dot product.
    T* X = A + nn;
    for (size_t e = tid; e < nn; e += nt) X[e] = 0;
    __syncthreads();
    for (int j = tid; j < nu; j += nt) {
      // P applied to e_j: follow the row swaps in factorisation order
      int r = j;
      for (int k = 0; k < nu; ++k) {
        if (piv[k] == r) r = k;
        else if (k == r) r = piv[k];
      }
      X[(size_t)r * nu + j] = 1;
    }
    __syncthreads();
    int G = 1;
    while (G < 32 && 2 * G * nu <= nt) G *= 2;
    const int sub = tid % G, cols = nt / G;
    for (int r = 1; r < nu; ++r) {                  // forward, unit lower
      for (int j0 = 0; j0 < nu; j0 += cols) {
        const int j = j0 + tid / G;
        T s = 0;
        if (j < nu)
          for (int c = sub; c < r; c += G) s += A[(size_t)r * nu + c] * X[(size_t)c * nu + j];
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, G);
        if (j < nu && sub == 0) X[(size_t)r * nu + j] -= s;
      }
      __syncthreads();
    }
    for (int r = nu - 1; r >= 0; --r) {             // backward
      for (int j0 = 0; j0 < nu; j0 += cols) {
        const int j = j0 + tid / G;
        T s = 0;
        if (j < nu)
          for (int c = r + 1 + sub; c < nu; c += G) s += A[(size_t)r * nu + c] * X[(size_t)c * nu + j];
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, G);
        if (j < nu && sub == 0) X[(size_t)r * nu + j] = (X[(size_t)r * nu + j] - s) / A[(size_t)r * nu + r];
      }
      __syncthreads();
    }
    for (size_t e = tid; e < nn; e += nt) inv[(e / nu) * ld + e % nu] = X[e];
    return;
  }
  // inverse from the factors in global memory (stride ld): solve L U x = P e_j, one warp per column
  const int lane = tid & 31, wid = tid >> 5, nw = nt / 32;
  for (int j = wid; j < nu; j += nw) {
    T* x = inv + (size_t)j;      // column j of the (row major, stride ld) inverse
    for (int r = lane; r < nu; r += 32) x[(size_t)r * ld] = (r == j) ? (T)1 : (T)0;
    __syncwarp();
    if (lane == 0)
      for (int k = 0; k < nu; ++k) {
        int p = piv[k];
        if (p != k) { T t = x[(size_t)k * ld]; x[(size_t)k * ld] = x[(size_t)p * ld]; x[(size_t)p * ld] = t; }
      }
    __syncwarp();
    for (int r = 0; r < nu; ++r) {                 // forward, unit lower
      T part = 0;
      for (int c = lane; c < r; c += 32) part += Ag[(size_t)r * ld + c] * x[(size_t)c * ld];
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) x[(size_t)r * ld] -= part;
      __syncwarp();
    }
    for (int r = nu - 1; r >= 0; --r) {            // backward
      T part = 0;
      for (int c = r + 1 + lane; c < nu; c += 32) part += Ag[(size_t)r * ld + c] * x[(size_t)c * ld];
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == 0) x[(size_t)r * ld] = (x[(size_t)r * ld] - part) / Ag[(size_t)r * ld + r];
      __syncwarp();
    }
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

// first level handled by the single-CTA tail: the first with at most kTailNodes nodes
static size_t tail_start(const Problem& P) {
  size_t l = 0;
  while (l + 1 < P.lv.size() && P.lv[l].g.N > kTailNodes) ++l;
  return l;
}
size_t mg_tail_start(const Problem& P) { return tail_start(P); }

// Parameters of the single-CTA tail over levels l0 .. end; *smem gets its shared
// memory bytes.  The irregular-row tables are staged in shared memory when the
// total stays within smem_limit (staging changes where they are read, not the result).
template <typename T>
TailParams<T> make_tail_params(Problem& P, size_t l0, T* u_out, size_t smem_limit, size_t* smem) {
  TailParams<T> tp;
  tp.u_out = u_out ? u_out : (T*)P.lv[l0].u;
  tp.nlev = (int)(P.lv.size() - l0);
  int off = 0;
  for (int k = 0; k < tp.nlev; ++k) {
    tp.L[k] = levk<T>(P.lv[l0 + k]);
    tp.off[k] = off;
    off += (int)P.lv[l0 + k].g.N;
  }
  tp.off[tp.nlev] = off;
  int toff = 0;
  for (int k = 0; k < tp.nlev; ++k) {
    const Level& L = P.lv[l0 + k];
    tp.toff[k] = toff;
    tp.tcount[k] = P.d_counts + 2 + (int)(l0 + k);
    tp.tcap[k] = L.irr_cap;
    toff += L.irr_cap * (2 * L.g.dim + 1);
  }
  tp.toff[tp.nlev] = toff;
  const size_t base = (sizeof(T) * 2 + 2 * sizeof(int)) * (size_t)off;   // u, f, aux, node coordinates
  tp.stage_tables = base + sizeof(T) * (size_t)toff <= smem_limit;
  if (!tp.stage_tables) {
    toff = 0;
    for (int k = 0; k <= tp.nlev; ++k) tp.toff[k] = 0;
  }
  tp.nu1 = P.opt.nu1;
  tp.nu2 = P.opt.nu2;
  tp.gamma = P.opt.cycle;
  tp.top_visits = 1;
  tp.neumann = P.desc.bc == IIM_BC_NEUMANN;
  tp.ld = P.coarse_n;
  tp.nu_dev = P.d_counts + kCountCoarse;
  tp.aug = P.aug;
  tp.map = P.coarse_map;
  tp.status = P.d_status + 1;
  const T* inv = (const T*)(sizeof(T) == 8 ? (void*)P.coarse_lu64 : (void*)P.coarse_lu32);
  tp.inv = inv + (size_t)P.coarse_n * P.coarse_n;
  tp.v = nullptr;
  tp.vscale = nullptr;
  tp.phase = P.phase;
  tp.inv_bp = (T)(1.0 / P.desc.beta_plus);
  tp.inv_bm = (T)(1.0 / P.desc.beta_minus);
  tp.z = nullptr;
  *smem = base + sizeof(T) * (size_t)toff;
  return tp;
}
template TailParams<float> make_tail_params<float>(Problem&, size_t, float*, size_t, size_t*);

// The tail entered from a finer level runs all gamma visits of its first level (they
// follow one another with the same right-hand side); from the finest level, one.
template <typename T>
static void launch_tail(Problem& P, size_t l0, const double* v, const double* vscale, double* z, cudaStream_t s,
                        T* u_out = nullptr) {
  size_t smem = 0;
  TailParams<T> tp = make_tail_params<T>(P, l0, u_out, 200 * 1024, &smem);
  tp.top_visits = l0 == 0 ? 1 : P.opt.cycle;
  tp.v = v;
  tp.vscale = vscale;
  tp.z = z;
  if (P.g.dim == 2) {
    if (smem > 48 * 1024) smem_optin((const void*)k_vcycle_tail<T, 2>);
    IIM_LAUNCH_PDL((k_vcycle_tail<T, 2>), 1, kTailThreads, smem, s, tp);
  } else {
    if (smem > 48 * 1024) smem_optin((const void*)k_vcycle_tail<T, 3>);
    IIM_LAUNCH_PDL((k_vcycle_tail<T, 3>), 1, kTailThreads, smem, s, tp);
  }
}

template <typename T, int TX, int TY>
static void launch_fine2d(Problem& P, size_t l, int mode, const double* v, const double* vscale, double* z,
                          const T* u_in, T* u_out, const T* uc, cudaStream_t s) {
  Fine2DParams<T> fp;
  fp.L = levk<T>(P.lv[l]);
  fp.u_in = u_in;
  fp.u_out = u_out;
  fp.uc = uc;
  if (l + 1 < P.lv.size()) fp.C = levk<T>(P.lv[l + 1]);
  fp.neumann = P.desc.bc == IIM_BC_NEUMANN;
  fp.v = v;
  fp.vscale = vscale;
  fp.phase = P.phase;
  fp.inv_bp = (T)(1.0 / P.desc.beta_plus);
  fp.inv_bm = (T)(1.0 / P.desc.beta_minus);
  fp.z = z;
  const int n = P.lv[l].g.n;
  dim3 grid(ceil_div(n, TX), ceil_div(n, TY));
  switch (mode) {
    case 0: IIM_LAUNCH((k_mg2d<T, TX, TY, 0>), grid, 256, 0, s, fp); break;
    case 1: IIM_LAUNCH((k_mg2d<T, TX, TY, 1>), grid, 256, 0, s, fp); break;
    case 2: IIM_LAUNCH((k_mg2d<T, TX, TY, 2>), grid, 256, 0, s, fp); break;
    case 3: IIM_LAUNCH((k_mg2d<T, TX, TY, 3>), grid, 256, 0, s, fp); break;
    case 5: IIM_LAUNCH((k_mg2d<T, TX, TY, 5>), grid, 256, 0, s, fp); break;
    case 6: IIM_LAUNCH((k_mg2d<T, TX, TY, 6>), grid, 256, 0, s, fp); break;
    case 7: IIM_LAUNCH((k_mg2d<T, TX, TY, 7>), grid, 256, 0, s, fp); break;
    default: IIM_LAUNCH((k_mg2d<T, TX, TY, 4>), grid, 256, 0, s, fp); break;
  }
}

// The red-black tile kernels (mg_rb.cuh) for the first visit's down (MODE 5) and up
// (MODE 6) steps of levels with at least kRbMinN cells per axis: NW warps of RW rows each.
constexpr int kRbMinN = 64;

template <typename T, int NW, int RW>
static void launch_rb(Problem& P, size_t l, int mode, const double* v, const double* vscale, double* z,
                      const T* u_in, T* u_out, const T* uc, cudaStream_t s) {
  const Level& L = P.lv[l];
  const Level& C = P.lv[l + 1];
  const LevelK<T> K = levk<T>(L);
  Rb2DParams<T> rp;
  rp.n = L.g.n;
  rp.nc = C.g.n;
  rp.ih2 = K.ih2;
  rp.inv_dreg = K.inv_dreg;
  rp.dreg = K.dreg;
  rp.cls = L.cls;
  rp.aux = L.aux;
  rp.tab = K.tab;
  rp.f_in = (const T*)L.f;
  rp.f_bf16 = L.f_bf16;
  rp.f_out = (T*)L.f;
  rp.v = mode == 5 ? v : nullptr;
  rp.vscale = vscale;
  rp.inv_bp = (T)(1.0 / P.desc.beta_plus);
  rp.inv_bm = (T)(1.0 / P.desc.beta_minus);
  rp.u_in = u_in;
  rp.u_out = u_out;
  rp.z = mode == 6 ? z : nullptr;
  rp.uc = uc;
  rp.cls_c = C.cls;
  rp.fc = (T*)C.f;
  rp.fc_bf16 = C.f_bf16;
  rp.neumann = P.desc.bc == IIM_BC_NEUMANN;
  constexpr int SY = NW * RW, TY = SY - 2 * kRbHalo;
  const dim3 grid(ceil_div(L.g.n, kRbTX), ceil_div(L.g.n, TY));
  if (mode == 5) {
    constexpr size_t sm = rb_smem_bytes<T, NW, RW, false>();
    if (sm > 48 * 1024) smem_optin((const void*)k_mg2d_rb<T, NW, RW, false>);
    IIM_LAUNCH_PDL((k_mg2d_rb<T, NW, RW, false>), grid, NW * 32, sm, s, rp);
  } else {
    constexpr size_t sm = rb_smem_bytes<T, NW, RW, true>();
    if (sm > 48 * 1024) smem_optin((const void*)k_mg2d_rb<T, NW, RW, true>);
    IIM_LAUNCH_PDL((k_mg2d_rb<T, NW, RW, true>), grid, NW * 32, sm, s, rp);
  }
}

template <typename T>
static void fine2d(Problem& P, size_t l, int mode, const double* v, const double* vscale, double* z, const T* u_in,
                   T* u_out, const T* uc, cudaStream_t s) {
  const int n = P.lv[l].g.n;
  if ((mode == 5 || mode == 6) && n >= kRbMinN) {
    // window heights measured best on GB300 (V-cycles of the 1024^2 and 2048^2 star problems):
    // 64 rows (512 threads) from 2048, 32 rows (512 threads) from 512, 16 rows (256 threads) below
    if (n >= 2048) launch_rb<T, 16, 4>(P, l, mode, v, vscale, z, u_in, u_out, uc, s);
    else if (n >= 512) launch_rb<T, 16, 2>(P, l, mode, v, vscale, z, u_in, u_out, uc, s);
    else launch_rb<T, 8, 2>(P, l, mode, v, vscale, z, u_in, u_out, uc, s);
    return;
  }
  if (n >= 512) launch_fine2d<T, 64, 16>(P, l, mode, v, vscale, z, u_in, u_out, uc, s);
  else launch_fine2d<T, 32, 8>(P, l, mode, v, vscale, z, u_in, u_out, uc, s);
}

// 2D: fused kernels per fine level (MODE 0, [4...], 1 down; 2, [4...], 3 up), ping-ponging
// between the level's two u buffers.  u0 is the level's starting u (the previous visit's
// result in a W-cycle; nullptr: zero).  Returns the buffer that holds the level's result.
template <typename T>
static T* vcycle2d(Problem& P, size_t l, size_t lt, const double* v, const double* vscale, double* z,
                   cudaStream_t s, const T* u0 = nullptr) {
  T* A = (T*)P.lv[l].u;
  T* B = (T*)P.lv[l].u2;
  if (l == lt) {
    launch_tail<T>(P, l, l == 0 ? v : nullptr, l == 0 ? vscale : nullptr, l == 0 ? z : nullptr, s, A);
    return A;
  }
  // gamma visits of the next level (one launch of the tail runs all of its own)
  auto coarser = [&]() -> const T* {
    if (l + 1 == lt) return vcycle2d<T>(P, l + 1, lt, nullptr, nullptr, nullptr, s);
    const T* uc = nullptr;
    for (int g = 0; g < P.opt.cycle; ++g) uc = vcycle2d<T>(P, l + 1, lt, nullptr, nullptr, nullptr, s, uc);
    return uc;
  };
  if (P.opt.nu1 == 2 && P.opt.nu2 == 2) {
    // two fused kernels per level: both pre-smoothing sweeps + restriction, then the
    // correction + both post-smoothing sweeps.  The result is in B, so a later visit
    // reads B and writes A.
    if (u0) fine2d<T>(P, l, 7, nullptr, nullptr, nullptr, u0, A, nullptr, s);
    else fine2d<T>(P, l, 5, l == 0 ? v : nullptr, vscale, nullptr, nullptr, A, nullptr, s);
    const T* uc = coarser();
    fine2d<T>(P, l, 6, nullptr, nullptr, l == 0 ? z : nullptr, A, B, uc, s);
    return B;
  }
  if (u0) fine2d<T>(P, l, 4, nullptr, nullptr, nullptr, u0, A, nullptr, s);
  else fine2d<T>(P, l, 0, l == 0 ? v : nullptr, vscale, nullptr, nullptr, A, nullptr, s);
  for (int it = 1; it < P.opt.nu1 - 1; ++it) {
    fine2d<T>(P, l, 4, nullptr, nullptr, nullptr, A, B, nullptr, s);
    std::swap(A, B);
  }
  fine2d<T>(P, l, 1, nullptr, nullptr, nullptr, A, B, nullptr, s);
  std::swap(A, B);
  const T* uc = coarser();
  fine2d<T>(P, l, 2, nullptr, nullptr, nullptr, A, B, uc, s);
  std::swap(A, B);
  for (int it = 1; it < P.opt.nu2 - 1; ++it) {
    fine2d<T>(P, l, 4, nullptr, nullptr, nullptr, A, B, nullptr, s);
    std::swap(A, B);
  }
  fine2d<T>(P, l, 3, nullptr, nullptr, l == 0 ? z : nullptr, A, B, nullptr, s);
  return B;
}

// generic path (3D fine levels): one kernel per half sweep, transfers separate; u is
// updated in place and starts from zero unless this is a later visit of a W-cycle
template <typename T>
static void vcycle(Problem& P, size_t l, size_t lt, cudaStream_t s, bool from_zero = true) {
  const int Tn = 256;
  Level& L = P.lv[l];
  T* u = (T*)L.u;
  T* f = (T*)L.f;
  if (l == lt) {
    launch_tail<T>(P, l, nullptr, nullptr, nullptr, s);
    return;
  }
  LevelView<T> V = view<T>(L);
  LevelK<T> K = levk<T>(L);
  const int64_t ncol = (L.g.N / L.g.n) * ((L.g.n + 1) / 2);
  if (from_zero) IIM_LAUNCH(k_zero<T>, ceil_div(L.g.N, Tn), Tn, 0, s, u, L.g.N);
  for (int it = 0; it < P.opt.nu1; ++it)
    for (int c = 0; c < 2; ++c)
      IIM_LAUNCH(k_smooth<T>, ceil_div(ncol, Tn), Tn, 0, s, V, K.ih2, K.dreg, u, f, L.f_bf16, c);
  Level& C = P.lv[l + 1];
  IIM_LAUNCH(k_resid_restrict<T>, ceil_div(C.g.N, Tn), Tn, 0, s, V, K.ih2, K.dreg, u, f, L.f_bf16, C.g, C.aux,
             (T*)C.f, C.f_bf16);
  if (l + 1 == lt) vcycle<T>(P, l + 1, lt, s);
  else
    for (int g = 0; g < P.opt.cycle; ++g) vcycle<T>(P, l + 1, lt, s, g == 0);
  IIM_LAUNCH(k_prolong<T>, ceil_div(L.g.N, Tn), Tn, 0, s, L.g, L.aux, u, C.g, C.aux, (const T*)C.u,
             P.desc.bc == IIM_BC_NEUMANN);
  for (int it = 0; it < P.opt.nu2; ++it)
    for (int c = 0; c < 2; ++c)
      IIM_LAUNCH(k_smooth<T>, ceil_div(ncol, Tn), Tn, 0, s, V, K.ih2, K.dreg, u, f, L.f_bf16, c);
}

template <typename T>
static void precondition_t(Problem& P, const double* v, const double* vscale, double* z, cudaStream_t s) {
  Level& L = P.lv[0];
  const int Tn = 256;
  const size_t lt = tail_start(P);
  if (lt == 0) {
    launch_tail<T>(P, 0, v, vscale, z, s);
    return;
  }
  if (P.g.dim == 2 && P.opt.nu1 >= 2 && P.opt.nu2 >= 2) {
    vcycle2d<T>(P, 0, lt, v, vscale, z, s);
    return;
  }
  IIM_LAUNCH(k_bridge_in<T>, ceil_div(L.g.N, Tn), Tn, 0, s, L.g, v, vscale, P.phase, L.aux,
             1.0 / P.desc.beta_plus, 1.0 / P.desc.beta_minus, (T*)L.f);
  vcycle<T>(P, 0, lt, s);
  IIM_LAUNCH(k_bridge_out<T>, ceil_div(L.g.N, Tn), Tn, 0, s, L.g, (const T*)L.u, z);
}

template <typename T>
static void smooth_fine_t(Problem& P, int colour, cudaStream_t s) {
  Level& L = P.lv[0];
  LevelView<T> V = view<T>(L);
  LevelK<T> K = levk<T>(L);
  const int64_t ncol = (L.g.N / L.g.n) * ((L.g.n + 1) / 2);
  IIM_LAUNCH(k_smooth<T>, ceil_div(ncol, 256), 256, 0, s, V, K.ih2, K.dreg, (T*)L.u, (const T*)L.f, L.f_bf16, colour);
}

// one red or black half sweep on the finest level (kernel timing)
void mg_smooth_fine(Problem& P, int colour, cudaStream_t s) {
  if (P.opt.mg_precision == IIM_MG_FP64) smooth_fine_t<double>(P, colour, s);
  else smooth_fine_t<float>(P, colour, s);
}

void mg_precondition(Problem& P, const double* v, const double* vscale, double* z, cudaStream_t s) {
  if (P.opt.mg_precision == IIM_MG_FP64) precondition_t<double>(P, v, vscale, z, s);
  else precondition_t<float>(P, v, vscale, z, s);
}

// The first level runs the fused down / up kernels (2D, V(2,2), above the tail)
bool mg_has_fused_first(const Problem& P) {
  return P.g.dim == 2 && tail_start(P) > 0 && P.opt.nu1 == 2 && P.opt.nu2 == 2;
}

// One kernel of the V-cycle alone (profiling): which 0 = the first level's down kernel,
// 1 = its up kernel (both need mg_has_fused_first), 2 = the coarse tail.
template <typename T>
static bool mg_one_kernel_t(Problem& P, int which, const double* v, double* z, cudaStream_t s) {
  const size_t lt = tail_start(P);
  if (which == 2) {
    launch_tail<T>(P, lt, lt == 0 ? v : nullptr, nullptr, lt == 0 ? z : nullptr, s);
    return true;
  }
  if (!mg_has_fused_first(P)) return false;
  T* A = (T*)P.lv[0].u;
  T* B = (T*)P.lv[0].u2;
  if (which == 0) fine2d<T>(P, 0, 5, v, nullptr, nullptr, nullptr, A, nullptr, s);
  else fine2d<T>(P, 0, 6, nullptr, nullptr, z, A, B, (const T*)P.lv[1].u, s);
  return true;
}

bool mg_one_kernel(Problem& P, int which, const double* v, double* z, cudaStream_t s) {
  if (P.opt.mg_precision == IIM_MG_FP64) return mg_one_kernel_t<double>(P, which, v, z, s);
  return mg_one_kernel_t<float>(P, which, v, z, s);
}

// coarse matrix, LU and inverse; coarse_lu{64,32} hold [A (cn*cn) | inverse (cn*cn)], cn the
// fixed size of the padded system (a re-run set-up with another geometry changes only the
// device-side unknown count)
void mg_coarse_factor(Problem& P, cudaStream_t s) {
  Level& C = P.lv.back();
  const int cn = P.coarse_n;
  if (cn <= 0) return;
  const int Tn = 256;
  IIM_LAUNCH(k_unknown_flag, ceil_div(C.g.N, Tn), Tn, 0, s, C.g, C.aux, C.flag);
  scan_exclusive(C.flag, C.idx, C.g.N, P.d_counts + kCountCoarse, P.scan_scratch, s);
  int32_t* inv = C.flag;            // reuse: node -> unknown index
  cudaMemsetAsync(P.coarse_map, 0xff, sizeof(int32_t) * (size_t)cn, s);    // -1: a slot no unknown uses
  IIM_LAUNCH(k_coarse_map, ceil_div(C.g.N, Tn), Tn, 0, s, C.g, C.aux, C.idx, P.coarse_map, inv);
  LevelView<double> V = view<double>(C);
  const int* nu = P.d_counts + kCountCoarse;
  // dynamic shared memory of the factorisation: room for the matrix and its inverse at the
  // unknown count of the creation's geometry with a quarter more (a later set-up with more
  // unknowns than that works on them in global memory instead); never more than the padded
  // system or 200 KB, so that small factorisations leave the SM to other kernels
  auto factor = [&](auto* A, auto* kernel, size_t esz) {
    const size_t nb = std::min((size_t)cn, (size_t)P.coarse_nu + P.coarse_nu / 4 + 8 + P.aug);
    size_t sm = std::min((size_t)2 * nb * nb * esz, (size_t)200 * 1024);
    smem_optin((const void*)kernel);
    IIM_LAUNCH(kernel, 1, 1024, sm, s, A, cn, nu, P.aug, P.coarse_piv, A + (size_t)cn * cn, P.d_status, sm / esz);
  };
  if (P.opt.mg_precision == IIM_MG_FP64) {
    IIM_LAUNCH(k_coarse_assemble<double>, ceil_div(cn, 128), 128, 0, s, V, P.coarse_map, nu, cn, inv, P.coarse_lu64,
               P.aug, P.d_status);
    factor(P.coarse_lu64, k_coarse_lu<double>, sizeof(double));
  } else {
    IIM_LAUNCH(k_coarse_assemble<float>, ceil_div(cn, 128), 128, 0, s, V, P.coarse_map, nu, cn, inv, P.coarse_lu32,
               P.aug, P.d_status);
    factor(P.coarse_lu32, k_coarse_lu<float>, sizeof(float));
  }
}


// ---------------------------------------------------------------------------- batched engine
// Grouped forms of the V-cycle kernels: each item is one block of the single-problem
// launch (a tile of the 2D fused kernels, 256 nodes of the 3D kernels, the whole
// tail), so a slot's V-cycle is the one its own solve would run.

__device__ __forceinline__ const double* eng_vj(const SlotDev& s) { return s.V + (size_t)s.j * s.Npad; }
__device__ __forceinline__ double* eng_zj(const SlotDev& s) { return s.Z + (size_t)s.j * s.Npad; }

template <int TX, int TY, int MODE>
__global__ void __launch_bounds__(256, 4) k_eng_mg2d(EngArgs A, int list, int d, int in_sel, int out_sel, int res_sel) {
  eng_for_items(A, list, [&](int si, int item) {
    const SlotDev& s = A.slots[si];
    if (s.role != kRoleIter) return;
    Fine2DParams<float> fp;
    fp.L = s.lev[d];
    fp.C = s.lev[d + 1 < s.nlev ? d + 1 : d];
    float* b0 = s.lev[d].u;
    float* b1 = s.u2[d];
    constexpr bool DOWN_FIRST = MODE == 0 || MODE == 5, UP_FIRST = MODE == 2 || MODE == 6;
    constexpr bool UP_LAST = MODE == 3 || MODE == 6;
    fp.u_in = DOWN_FIRST ? nullptr : (in_sel ? b1 : b0);
    fp.u_out = out_sel ? b1 : b0;
    fp.uc = nullptr;
    if (UP_FIRST) fp.uc = (d + 1 < s.nfine && res_sel) ? s.u2[d + 1] : s.lev[d + 1].u;
    fp.neumann = s.neumann;
    fp.v = (DOWN_FIRST && d == 0) ? eng_vj(s) : nullptr;
    fp.vscale = &s.sc->inv_norm[s.j];
    fp.phase = s.phase;
    fp.inv_bp = s.inv_bp;
    fp.inv_bm = s.inv_bm;
    fp.z = (UP_LAST && d == 0) ? eng_zj(s) : nullptr;
    const int gx = (s.lev[d].n + TX - 1) / TX;
    mg2d_tile<float, TX, TY, MODE>(fp, item % gx, item / gx);
  });
}

__global__ void __launch_bounds__(kTailThreads) k_eng_tail(EngArgs A) {
  eng_for_items(A, kListTail, [&](int si, int) {
    const SlotDev& s = A.slots[si];
    if (s.role != kRoleIter) return;
    const bool top = s.nfine == 0;
    if (s.dim == 2)
      vcycle_tail_body<float, 2>(s.tail, top ? eng_vj(s) : nullptr, top ? &s.sc->inv_norm[s.j] : nullptr,
                            top ? eng_zj(s) : nullptr);
    else
      vcycle_tail_body<float, 3>(s.tail, top ? eng_vj(s) : nullptr, top ? &s.sc->inv_norm[s.j] : nullptr,
                            top ? eng_zj(s) : nullptr);
  });
}

__device__ __forceinline__ LevelView<float> eng_view(const SlotDev& s, int d) {
  LevelView<float> v;
  v.g.dim = s.lev[d].dim;
  v.g.n = s.lev[d].n;
  v.g.N = s.lev[d].N;
  v.g.h = 2.0 / s.lev[d].n;
  v.aux = s.lev[d].aux;
  v.tab = s.lev[d].tab;
  return v;
}

// 3D kernels, kind: 0 bridge in, 1 zero, 2 smooth, 3 residual + restriction, 4 prolongation, 5 bridge out
template <int KIND>
__global__ void __launch_bounds__(256) k_eng_mg3d(EngArgs A, int list, int d, int colour) {
  eng_for_items(A, list, [&](int si, int item) {
    const SlotDev& s = A.slots[si];
    if (s.role != kRoleIter) return;
    const int64_t i = (int64_t)item * 256 + threadIdx.x;
    const LevelK<float>& K = s.lev[d];
    const LevelView<float> V = eng_view(s, d);
    if (KIND == 0) {
      bridge_in_body<float>(V.g, eng_vj(s), &s.sc->inv_norm[s.j], s.phase, K.aux, 1.0 / s.GP.beta_p,
                            1.0 / s.GP.beta_m, K.f, i);
    } else if (KIND == 1) {
      if (i < K.N) K.u[i] = 0.f;
    } else if (KIND == 2) {
      smooth_body<float>(V, K.ih2, K.dreg, K.u, K.f, K.f_bf16, colour, i);
    } else if (KIND == 3) {
      const LevelView<float> C = eng_view(s, d + 1);
      resid_restrict_body<float>(V, K.ih2, K.dreg, K.u, K.f, K.f_bf16, C.g, C.aux, s.lev[d + 1].f, i,
                                 s.lev[d + 1].f_bf16);
    } else if (KIND == 4) {
      const LevelView<float> C = eng_view(s, d + 1);
      prolong_body<float>(V.g, K.aux, K.u, C.g, C.aux, s.lev[d + 1].u, s.neumann, i);
    } else {
      if (i < K.N) eng_zj(s)[i] = (double)K.u[i];
    }
  });
}

void eng_mg2d_tile_items(int n, int shape, int* gx, int* gy) {
  *gx = ceil_div(n, kShapeTX[shape]);
  *gy = ceil_div(n, kShapeTY[shape]);
}

template <int TX, int TY>
static void launch_eng_mg2d(const EngArgs& A, const EngMgStep& st, cudaStream_t s) {
  const int list = kListMg2d + st.depth * kEngShapes + st.shape;
#define IIM_ENG_MG2D(MODE)                                                                                     \
  IIM_LAUNCH((k_eng_mg2d<TX, TY, MODE>), eng_grid((const void*)k_eng_mg2d<TX, TY, MODE>, 256, 0), 256, 0, s, A, \
             list, st.depth, st.in_sel, st.out_sel, st.res_sel)
  switch (st.mode) {
    case 0: IIM_ENG_MG2D(0); break;
    case 1: IIM_ENG_MG2D(1); break;
    case 2: IIM_ENG_MG2D(2); break;
    case 3: IIM_ENG_MG2D(3); break;
    case 5: IIM_ENG_MG2D(5); break;
    case 6: IIM_ENG_MG2D(6); break;
    default: IIM_ENG_MG2D(4); break;
  }
#undef IIM_ENG_MG2D
}

void eng_launch_mg(const EngArgs& A, const EngMgStep& st, size_t tail_smem, cudaStream_t s) {
  if (st.kind == 0) {
    switch (st.shape) {
      case 0: launch_eng_mg2d<32, 8>(A, st, s); break;
      case 1: launch_eng_mg2d<64, 8>(A, st, s); break;
      case 2: launch_eng_mg2d<32, 16>(A, st, s); break;
      default: launch_eng_mg2d<64, 16>(A, st, s); break;
    }
    return;
  }
  if (st.kind == 1) {
    smem_optin((const void*)k_eng_tail);
    IIM_LAUNCH(k_eng_tail, eng_grid((const void*)k_eng_tail, kTailThreads, tail_smem), kTailThreads, tail_smem, s, A);
    return;
  }
  const int k3 = st.kind - 2;
  const int d = st.depth;
#define IIM_ENG_MG3D(KIND, LIST)                                                                             \
  IIM_LAUNCH(k_eng_mg3d<KIND>, eng_grid((const void*)k_eng_mg3d<KIND>, 256, 0), 256, 0, s, A, LIST, d, st.colour)
  switch (k3) {
    case 0: IIM_ENG_MG3D(0, kList3dN + 0); break;
    case 1: IIM_ENG_MG3D(1, kList3dN + d); break;
    case 2: IIM_ENG_MG3D(2, kList3dCol + d); break;
    case 3: IIM_ENG_MG3D(3, kList3dCoarse + d); break;
    case 4: IIM_ENG_MG3D(4, kList3dN + d); break;
    default: IIM_ENG_MG3D(5, kList3dN + 0); break;
  }
#undef IIM_ENG_MG3D
}

}  // namespace iim
