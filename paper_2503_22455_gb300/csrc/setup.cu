// Device set-up of one problem: phases, control points, curvature check,
// affected-node records, least-squares fits (paper Sec. 2.1-2.2) and the
// Shortley-Weller levels of the multigrid preconditioner (Sec. 3.1, 3.3).
#include "kernels.cuh"

namespace iim {

__device__ inline void node_index(const GridView& g, int64_t i, int* m) {
  m[0] = (int)(i % g.n);
  int64_t r = i / g.n;
  m[1] = (int)(r % g.n);
  m[2] = g.dim > 2 ? (int)(r / g.n) : 0;
}
__device__ inline double node_x(const GridView& g, int m) { return -1.0 + ((double)m + 0.5) * g.h; }
__device__ inline int64_t stride_of(const GridView& g, int ax) {
  return ax == 0 ? 1 : (ax == 1 ? (int64_t)g.n : (int64_t)g.n * g.n);
}

// ------------------------------------------------------------------------------ phase
__global__ void k_phase(Geom G, GridView g, uint8_t* __restrict__ phase) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int m[3];
  node_index(g, i, m);
  double x[3] = {node_x(g, m[0]), node_x(g, m[1]), g.dim > 2 ? node_x(g, m[2]) : 0.0};
  phase[i] = phase_plus_at(G, x) ? 1 : 0;
}

// flag[ax * N + i] = 1 if the edge (i, i + e_ax) joins nodes of different phase
__global__ void k_edge_flags(GridView g, const uint8_t* __restrict__ phase, int32_t* __restrict__ flag) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.N * g.dim) return;
  int ax = (int)(e / g.N);
  int64_t i = e - (int64_t)ax * g.N;
  int m[3];
  node_index(g, i, m);
  int f = 0;
  if (m[ax] < g.n - 1) f = phase[i] != phase[i + stride_of(g, ax)];
  flag[e] = f;
}

// cut edges -> compact list in canonical order (axis, lower node)
__global__ void k_compact(const int32_t* __restrict__ flag, const int32_t* __restrict__ id, int64_t len, int cap,
                          int32_t* __restrict__ list, int* status) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len || !flag[e]) return;
  int c = id[e];
  if (c >= cap) {
    set_status(status, IIM_ERR_CAPACITY);
    return;
  }
  list[c] = (int32_t)e;
}

// one thread per control point, so that the FP64 root solves run on full warps
__global__ void k_crossings(Geom G, GridView g, const int32_t* __restrict__ edges, const int* __restrict__ K, int cap,
                            const uint8_t* __restrict__ phase, int32_t* cr_axis, int32_t* cr_lo,
                            uint8_t* cr_loplus, double* cr_t, double* cr_x, double* cr_n, double* cr_kappa,
                            int* status) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= *K || c >= cap) return;
  const int64_t e = edges[c];
  int ax = (int)(e / g.N);
  int64_t i = e - (int64_t)ax * g.N;
  int m[3];
  node_index(g, i, m);
  double x0[3] = {node_x(g, m[0]), node_x(g, m[1]), g.dim > 2 ? node_x(g, m[2]) : 0.0};
  double t = edge_root(G, x0, ax, g.h, g.dim);
  double x[3] = {x0[0], x0[1], x0[2]};
  x[ax] += t * g.h;
  double gr[3] = {0, 0, 0};
  geom_grad_g(G, x, gr);
  double gn = 0;
  for (int k = 0; k < g.dim; ++k) gn += gr[k] * gr[k];
  gn = sqrt(gn);
  cr_axis[c] = ax;
  cr_lo[c] = (int32_t)i;
  cr_loplus[c] = phase[i];
  cr_t[c] = t;
  for (int k = 0; k < g.dim; ++k) {
    cr_x[c * g.dim + k] = x[k];
    cr_n[c * g.dim + k] = -G.sign * gr[k] / gn;   // n = -grad(phi)/|grad(phi)|
  }
  cr_kappa[c] = geom_curvature(G, x);
}

__global__ void k_curvature_check(const double* __restrict__ kappa, const int* __restrict__ K, double h, int* status) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < *K && kappa[c] * h >= 0.25) set_status(status, IIM_ERR_CURVATURE);
}

// ------------------------------------------------------------------------------ affected nodes
struct WalkParams {
  GridView g;
  int w, q, interface_, box_bc;
};

__device__ inline bool is_unknown(const WalkParams& P, uint8_t ph) { return P.interface_ || ph; }

// geometry checks + affected flag per node
__global__ void k_affected_flags(WalkParams P, const uint8_t* __restrict__ phase, int32_t* __restrict__ flag,
                                 int* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const GridView& g = P.g;
  if (i >= g.N) return;
  int m[3];
  node_index(g, i, m);
  uint8_t ph = phase[i];
  bool unk = is_unknown(P, ph);
  // distance to the box along any axis
  int dmin = g.n;
  for (int k = 0; k < g.dim; ++k) dmin = min(dmin, min(m[k], g.n - 1 - m[k]));
  if (P.box_bc == IIM_BOX_DIRICHLET) {
    if (dmin < P.q + 1 + P.w && !ph) set_status(status, IIM_ERR_GEOMETRY);
  } else if (unk && dmin < P.w) {
    set_status(status, IIM_ERR_GEOMETRY);
  }
  int f = 0;
  if (unk) {
    for (int ax = 0; ax < g.dim && !f; ++ax) {
      int64_t st = stride_of(g, ax);
      for (int s = -1; s <= 1 && !f; s += 2) {
        for (int j = 1; j <= P.w; ++j) {
          int pos = m[ax] + j * s;
          if (pos < 0 || pos >= g.n) { f = 1; break; }
          if (phase[i + j * s * st] != ph) { f = 1; break; }
        }
      }
    }
  }
  flag[i] = f;
}

__global__ void k_affected_fill(WalkParams P, const uint8_t* __restrict__ phase, const int32_t* __restrict__ flag,
                                const int32_t* __restrict__ idx, const int32_t* __restrict__ edge_id, int cap,
                                int32_t* aff_node, int32_t* aff_fit, int32_t* aff_j, int* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const GridView& g = P.g;
  if (i >= g.N || !flag[i]) return;
  int a = idx[i];
  if (a >= cap) {
    set_status(status, IIM_ERR_CAPACITY);
    return;
  }
  int m[3];
  node_index(g, i, m);
  uint8_t ph = phase[i];
  aff_node[a] = (int32_t)i;
  for (int ax = 0; ax < g.dim; ++ax) {
    int64_t st = stride_of(g, ax);
    for (int sd = 0; sd < 2; ++sd) {
      int s = sd ? 1 : -1;
      int fit = -1, js = 0;
      for (int j = 1; j <= P.w; ++j) {
        int pos = m[ax] + j * s;
        if (pos < 0 || pos >= g.n) { fit = -2; js = j; break; }
        int64_t nb = i + j * s * st;
        if (phase[nb] != ph) {
          int64_t lower = s > 0 ? nb - st : nb;       // edge between offsets j-1 and j
          int c = edge_id[(int64_t)ax * g.N + lower];
          fit = P.interface_ ? 2 * c + (ph ? 0 : 1) : c;
          js = j;
          break;
        }
      }
      aff_fit[a * 2 * g.dim + 2 * ax + sd] = fit;
      aff_j[a * 2 * g.dim + 2 * ax + sd] = js;
    }
  }
}

// ------------------------------------------------------------------------------ least-squares fits
struct FitParams {
  GridView g;
  int q, w, M, rcap, bc, interface_;
  double beta_p;
  const uint8_t* phase;
  const int32_t* cr_axis;
  const int32_t* cr_lo;
  const uint8_t* cr_loplus;
  const double* cr_t;
  const double* cr_x;
  const double* cr_n;
  const int* monos;                       // [M][3]
  const int* K;                           // device count of crossings
  int32_t* fit_R;
  int32_t* fit_nodes;
  double* fit_coef;
  double* fit_cdat;
  int* status;
};

constexpr int kFitThreads = 256;

__device__ inline double monomial(const int* e, const double* xi, int dim) {
  double v = 1.0;
  for (int k = 0; k < dim; ++k)
    for (int p = 0; p < e[k]; ++p) v *= xi[k];
  return v;
}

// lexicographic minimum of (d2, flat)
__device__ inline void better(double& d2, int& fl, double od2, int ofl) {
  if (od2 < d2 || (od2 == d2 && ofl < fl)) { d2 = od2; fl = ofl; }
}

// One CTA per fit: gather X_c, scaled-monomial Vandermonde, Householder QR,
// ghost / derivative rows v^T R^-1 Q^T (Sec. 2.1: one QR per control point,
// one triangular solve and one product per stencil).
__global__ void __launch_bounds__(kFitThreads) k_fit(FitParams P, const int* __restrict__ only) {
  extern __shared__ double sm[];
  const int f = blockIdx.x;
  const GridView& g = P.g;
  const int c = P.interface_ ? (f >> 1) : f;
  if (c >= *P.K) return;
  if (only && !only[f]) return;
  const bool sig_plus = P.interface_ ? ((f & 1) == 0) : true;
  const int d = g.dim, n = g.n, M = P.M, LD = P.rcap + 1;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double* V = sm;                         // [M][LD] column major
  double* S = V + (size_t)M * LD;         // [4][LD] stencil rows
  double* Y = S + 4 * LD;                 // [4][M]
  double* alpha = Y + 4 * M;              // [M]
  double* beta = alpha + M;               // [M]
  double* rel = beta + M;                 // [rcap][3]
  int* nodes = (int*)(rel + 3 * P.rcap);  // [rcap]
  __shared__ int cnt[kFitThreads];
  __shared__ double red_d[kFitThreads / 32];
  __shared__ int red_i[kFitThreads / 32];
  __shared__ int sR, s_near, s_ok;

  double xc[3] = {0, 0, 0}, nrm[3] = {0, 0, 0};
  for (int k = 0; k < d; ++k) {
    xc[k] = P.cr_x[c * d + k];
    nrm[k] = P.cr_n[c * d + k];
  }
  double ns[3];
  for (int k = 0; k < 3; ++k) ns[k] = sig_plus ? -nrm[k] : nrm[k];   // points into phase sigma
  const int ax = P.cr_axis[c];
  const int64_t lo = P.cr_lo[c];
  const bool lo_sig = (P.cr_loplus[c] != 0) == sig_plus;
  int cidx[3];
  for (int k = 0; k < 3; ++k) cidx[k] = k < d ? (int)floor((xc[k] + 1.0) / g.h - 0.5) : 0;

  for (int grow = 0; grow <= 3; ++grow) {
    const double an = P.q + 1.0 + 0.5 * grow, at = P.q / 2 + 1.0 + 0.5 * grow;
    const int rad = (int)ceil(an) + 1;
    int wlo[3] = {0, 0, 0}, wext[3] = {1, 1, 1};
    for (int k = 0; k < d; ++k) {
      wlo[k] = max(0, cidx[k] - rad);
      wext[k] = min(n, cidx[k] + rad + 2) - wlo[k];
    }
    const int total = wext[0] * wext[1] * wext[2];
    // pass 1: phase-sigma node nearest to x_c
    double bd = 1e300;
    int bf = 0x7fffffff;
    for (int p = tid; p < total; p += kFitThreads) {
      int i0 = p % wext[0], r = p / wext[0], i1 = r % wext[1], i2 = r / wext[1];
      int mm[3] = {wlo[0] + i0, wlo[1] + i1, wlo[2] + i2};
      int64_t fl = mm[0] + (int64_t)n * mm[1] + (int64_t)n * n * mm[2];
      if ((P.phase[fl] != 0) != sig_plus) continue;
      double d2 = 0;
      for (int k = 0; k < d; ++k) {
        double rr = (node_x(g, mm[k]) - xc[k]) / g.h;
        d2 += rr * rr;
      }
      better(bd, bf, d2, (int)fl);
    }
    for (int o = 16; o > 0; o >>= 1) {
      double od = __shfl_xor_sync(0xffffffffu, bd, o);
      int of = __shfl_xor_sync(0xffffffffu, bf, o);
      better(bd, bf, od, of);
    }
    if (lane == 0) { red_d[wid] = bd; red_i[wid] = bf; }
    __syncthreads();
    if (tid == 0) {
      double b0 = red_d[0];
      int f0 = red_i[0];
      for (int k = 1; k < kFitThreads / 32; ++k) better(b0, f0, red_d[k], red_i[k]);
      s_near = f0;
    }
    __syncthreads();
    const int nearest = s_near;
    // pass 2: ordered compaction of the half-ellipse nodes
    const int chunk = (total + kFitThreads - 1) / kFitThreads;
    const int p0 = tid * chunk, p1 = min(total, p0 + chunk);
    auto selected = [&](int p, int64_t& fl, double* rr) -> bool {
      int i0 = p % wext[0], r = p / wext[0], i1 = r % wext[1], i2 = r / wext[1];
      int mm[3] = {wlo[0] + i0, wlo[1] + i1, wlo[2] + i2};
      fl = mm[0] + (int64_t)n * mm[1] + (int64_t)n * n * mm[2];
      if ((P.phase[fl] != 0) != sig_plus || fl == nearest) return false;
      double d2 = 0, t = 0;
      for (int k = 0; k < d; ++k) {
        rr[k] = (node_x(g, mm[k]) - xc[k]) / g.h;
        d2 += rr[k] * rr[k];
        t += rr[k] * ns[k];
      }
      double tau2 = fmax(d2 - t * t, 0.0);
      return t >= 0.0 && tau2 / (at * at) + t * t / (an * an) <= 1.0;
    };
    int my = 0;
    for (int p = p0; p < p1; ++p) {
      int64_t fl;
      double rr[3];
      my += selected(p, fl, rr);
    }
    cnt[tid] = my;
    __syncthreads();
    if (tid == 0) {
      int acc = 0;
      for (int k = 0; k < kFitThreads; ++k) { int v = cnt[k]; cnt[k] = acc; acc += v; }
      sR = acc;
    }
    __syncthreads();
    const int R = sR;
    if (R > P.rcap) {
      if (tid == 0) set_status(P.status, IIM_ERR_CAPACITY);
      return;
    }
    {
      int o = cnt[tid];
      for (int p = p0; p < p1; ++p) {
        int64_t fl;
        double rr[3] = {0, 0, 0};
        if (selected(p, fl, rr)) {
          nodes[o] = (int)fl;
          for (int k = 0; k < 3; ++k) rel[o * 3 + k] = rr[k];
          ++o;
        }
      }
    }
    __syncthreads();
    const int m = R + 1;
    if (m < M) continue;
    // Vandermonde: row 0 is the control point (xi = 0)
    for (int e = tid; e < m * M; e += kFitThreads) {
      int col = e / m, row = e - col * m;
      double v;
      if (row == 0) v = col == 0 ? 1.0 : 0.0;
      else v = monomial(P.monos + 3 * col, rel + 3 * (row - 1), d);
      V[(size_t)col * LD + row] = v;
    }
    __syncthreads();
    // Householder QR
    for (int k = 0; k < M; ++k) {
      if (wid == 0) {
        double s = 0;
        for (int r = k + lane; r < m; r += 32) s += V[(size_t)k * LD + r] * V[(size_t)k * LD + r];
        s = warp_sum(s);
        if (lane == 0) {
          double x0 = V[(size_t)k * LD + k];
          double nr = sqrt(s);
          double a = x0 >= 0 ? -nr : nr;
          double vtv = 2.0 * (s - x0 * a);
          V[(size_t)k * LD + k] = x0 - a;
          alpha[k] = a;
          beta[k] = vtv > 0 ? 2.0 / vtv : 0.0;
        }
      }
      __syncthreads();
      for (int j = k + 1 + wid; j < M; j += kFitThreads / 32) {
        double s = 0;
        for (int r = k + lane; r < m; r += 32) s += V[(size_t)k * LD + r] * V[(size_t)j * LD + r];
        s = warp_sum(s) * beta[k];
        for (int r = k + lane; r < m; r += 32) V[(size_t)j * LD + r] -= s * V[(size_t)k * LD + r];
      }
      __syncthreads();
    }
    if (tid == 0) {
      double mx = 0, mn = 1e300;
      for (int k = 0; k < M; ++k) { mx = fmax(mx, fabs(alpha[k])); mn = fmin(mn, fabs(alpha[k])); }
      s_ok = (mn >= 1e-8 * mx) && mx > 0;
    }
    __syncthreads();
    if (!s_ok) continue;
    // stencil rows: warp t < w -> ghost t, warp w -> normal derivative (n out of Omega+)
    const int nt = P.w + 1;                // ghosts and the normal derivative (every condition)
    if (wid < nt) {
      double* y = Y + wid * M;
      double* s = S + wid * LD;
      if (wid < P.w) {
        // ghost node: first node past the crossing, away from the sigma side
        int step = lo_sig ? 1 : -1;
        int mlo[3];
        {
          int64_t r = lo;
          mlo[0] = (int)(r % n); r /= n; mlo[1] = (int)(r % n); mlo[2] = d > 2 ? (int)(r / n) : 0;
        }
        int gm[3] = {mlo[0], mlo[1], mlo[2]};
        gm[ax] += (lo_sig ? 1 : 0) + wid * step;
        double xi[3] = {0, 0, 0};
        for (int k = 0; k < d; ++k) xi[k] = (node_x(g, gm[k]) - xc[k]) / g.h;
        for (int col = lane; col < M; col += 32) y[col] = monomial(P.monos + 3 * col, xi, d);
      } else {
        for (int col = lane; col < M; col += 32) {
          const int* e = P.monos + 3 * col;
          int deg = e[0] + e[1] + e[2];
          double v = 0;
          if (deg == 1) for (int k = 0; k < d; ++k) if (e[k] == 1) v = nrm[k] / g.h;
          y[col] = v;
        }
      }
      __syncwarp();
      // y = R^-T c  (R[l][i] = V[i][l] for l < i)
      for (int i = 0; i < M; ++i) {
        double part = 0;
        for (int l = lane; l < i; l += 32) part += V[(size_t)i * LD + l] * y[l];
        part = warp_sum(part);
        if (lane == 0) y[i] = (y[i] - part) / alpha[i];
        __syncwarp();
      }
      // s = Q [y; 0] = H_0 H_1 ... H_{M-1} [y; 0]
      for (int r = lane; r < m; r += 32) s[r] = r < M ? y[r] : 0.0;
      __syncwarp();
      for (int k = M - 1; k >= 0; --k) {
        double dot = 0;
        for (int r = k + lane; r < m; r += 32) dot += V[(size_t)k * LD + r] * s[r];
        dot = warp_sum(dot) * beta[k];
        for (int r = k + lane; r < m; r += 32) s[r] -= dot * V[(size_t)k * LD + r];
        __syncwarp();
      }
    }
    __syncthreads();
    // outputs
    const int rows = P.w + 1;
    double* coef = P.fit_coef + (size_t)f * rows * P.rcap;
    double* cdat = P.fit_cdat + (size_t)f * rows;
    if (P.bc == IIM_BC_NEUMANN) {
      // fold u_c = (qbar - sum D_i u_i) / D_c into the ghost rows, D = beta+ * derivative row (Eqs. 5-6)
      __shared__ double s_dn;
      if (wid == 0) {
        double s2 = 0;
        for (int r = lane; r < m; r += 32) { double v = P.beta_p * S[P.w * LD + r]; s2 += v * v; }
        s2 = warp_sum(s2);
        if (lane == 0) s_dn = sqrt(s2);
      }
      __syncthreads();
      const double Dc = P.beta_p * S[P.w * LD + 0];
      if (!(fabs(Dc) >= 1e-12 * s_dn)) {
        if (tid == 0) set_status(P.status, IIM_ERR_SINGULAR);
        return;
      }
      for (int e = tid; e < P.w * R; e += kFitThreads) {
        int k = e / R, al = e - k * R;
        coef[(size_t)k * P.rcap + al] = S[k * LD + 1 + al] - S[k * LD] * (P.beta_p * S[P.w * LD + 1 + al]) / Dc;
      }
      if (tid < P.w) cdat[tid] = S[tid * LD] / Dc;
      // row w: the control value itself, u_c = (qbar - sum D_i u_i) / D_c (Eq. 6)
      for (int e = tid; e < R; e += kFitThreads) coef[(size_t)P.w * P.rcap + e] = -(P.beta_p * S[P.w * LD + 1 + e]) / Dc;
      if (tid == 0) cdat[P.w] = 1.0 / Dc;
    } else {
      for (int e = tid; e < nt * R; e += kFitThreads) {
        int k = e / R, al = e - k * R;
        coef[(size_t)k * P.rcap + al] = S[k * LD + 1 + al];
      }
      if (tid < nt) cdat[tid] = S[tid * LD];
    }
    for (int e = tid; e < R; e += kFitThreads) P.fit_nodes[(size_t)f * P.rcap + e] = nodes[e];
    if (tid == 0) P.fit_R[f] = R;
    return;
  }
  if (tid == 0) set_status(P.status, IIM_ERR_RANK);
}

// One warp per fit (the common case): rows of X_c up to RW; fits with more rows are
// flagged in `overflow` and redone by k_fit (one CTA each).  Householder QR with
// lanes over columns (the Householder vector is broadcast from shared memory),
// then the w (+1) stencil rows by quarter-warps, one row each.
struct WarpFitSmem {
  int RW, LDW, M;
  __host__ __device__ size_t bytes() const {
    return sizeof(double) * ((size_t)M * LDW + 4 * LDW + 4 * M + 2 * M + 3 * RW) + sizeof(int) * RW;
  }
};

__device__ inline void qw_sum(double& v) {          // sum over the 8 lanes of a quarter-warp
  v += __shfl_xor_sync(0xffffffffu, v, 4, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 2, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 1, 8);
}

__global__ void __launch_bounds__(128) k_fit_warp(FitParams P, WarpFitSmem L, int* __restrict__ overflow) {
  extern __shared__ double smw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int f = blockIdx.x * (blockDim.x >> 5) + wib;
  const GridView& g = P.g;
  const int nfit_here = P.interface_ ? 2 * (*P.K) : *P.K;
  if (f >= nfit_here) return;
  const int c = P.interface_ ? (f >> 1) : f;
  const bool sig_plus = P.interface_ ? ((f & 1) == 0) : true;
  const int d = g.dim, n = g.n, M = P.M, LDW = L.LDW, RW = L.RW;
  double* V = smw + (size_t)wib * (L.bytes() / sizeof(double) + 1);
  double* S = V + (size_t)M * LDW;         // [4][LDW]
  double* Y = S + 4 * LDW;                 // [4][M]
  double* alpha = Y + 4 * M;               // [M] (stores 1/R_kk after the rank test)
  double* beta = alpha + M;                // [M]
  double* rel = beta + M;                  // [RW][3]
  int* nodes = (int*)(rel + 3 * RW);       // [RW]
  double xc[3] = {0, 0, 0}, nrm[3] = {0, 0, 0};
  for (int k = 0; k < d; ++k) {
    xc[k] = P.cr_x[c * d + k];
    nrm[k] = P.cr_n[c * d + k];
  }
  double ns[3];
  for (int k = 0; k < 3; ++k) ns[k] = sig_plus ? -nrm[k] : nrm[k];
  const int ax = P.cr_axis[c];
  const int64_t lo = P.cr_lo[c];
  const bool lo_sig = (P.cr_loplus[c] != 0) == sig_plus;
  int cidx[3];
  for (int k = 0; k < 3; ++k) cidx[k] = k < d ? (int)floor((xc[k] + 1.0) / g.h - 0.5) : 0;
  for (int grow = 0; grow <= 3; ++grow) {
    const double an = P.q + 1.0 + 0.5 * grow, at = P.q / 2 + 1.0 + 0.5 * grow;
    const int rad = (int)ceil(an) + 1;
    int wlo[3] = {0, 0, 0}, wext[3] = {1, 1, 1};
    for (int k = 0; k < d; ++k) {
      wlo[k] = max(0, cidx[k] - rad);
      wext[k] = min(n, cidx[k] + rad + 2) - wlo[k];
    }
    const int total = wext[0] * wext[1] * wext[2];
    auto position = [&](int p, int* mm) {
      const int i0 = p % wext[0], r = p / wext[0];
      mm[0] = wlo[0] + i0;
      mm[1] = wlo[1] + r % wext[1];
      mm[2] = wlo[2] + r / wext[1];
    };
    // nearest phase-sigma node
    double bd = 1e300;
    int bf = 0x7fffffff;
    for (int p = lane; p < total; p += 32) {
      int mm[3];
      position(p, mm);
      const int64_t fl = mm[0] + (int64_t)n * mm[1] + (int64_t)n * n * mm[2];
      if ((P.phase[fl] != 0) != sig_plus) continue;
      double d2 = 0;
      for (int k = 0; k < d; ++k) {
        const double rr = (node_x(g, mm[k]) - xc[k]) / g.h;
        d2 += rr * rr;
      }
      better(bd, bf, d2, (int)fl);
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double od = __shfl_xor_sync(0xffffffffu, bd, o);
      const int of = __shfl_xor_sync(0xffffffffu, bf, o);
      better(bd, bf, od, of);
    }
    const int nearest = bf;
    auto selected = [&](int p, int64_t& fl, double* rr) -> bool {
      int mm[3];
      position(p, mm);
      fl = mm[0] + (int64_t)n * mm[1] + (int64_t)n * n * mm[2];
      if ((P.phase[fl] != 0) != sig_plus || fl == nearest) return false;
      double d2 = 0, t = 0;
      for (int k = 0; k < d; ++k) {
        rr[k] = (node_x(g, mm[k]) - xc[k]) / g.h;
        d2 += rr[k] * rr[k];
        t += rr[k] * ns[k];
      }
      const double tau2 = fmax(d2 - t * t, 0.0);
      return t >= 0.0 && tau2 / (at * at) + t * t / (an * an) <= 1.0;
    };
    // ordered compaction: contiguous chunks per lane, warp prefix sum of the counts
    const int chunk = (total + 31) / 32;
    const int p0 = lane * chunk, p1 = min(total, p0 + chunk);
    int my = 0;
    for (int p = p0; p < p1; ++p) {
      int64_t fl;
      double rr[3];
      my += selected(p, fl, rr);
    }
    int incl = my;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int R = __shfl_sync(0xffffffffu, incl, 31);
    if (R > RW) {
      if (lane == 0) overflow[f] = 1;
      return;
    }
    {
      int o = incl - my;
      for (int p = p0; p < p1; ++p) {
        int64_t fl;
        double rr[3] = {0, 0, 0};
        if (selected(p, fl, rr)) {
          nodes[o] = (int)fl;
          for (int k = 0; k < 3; ++k) rel[o * 3 + k] = rr[k];
          ++o;
        }
      }
    }
    __syncwarp();
    const int m = R + 1;
    if (m < M) continue;
    for (int e = lane; e < m * M; e += 32) {
      const int col = e / m, row = e - col * m;
      V[(size_t)col * LDW + row] = row == 0 ? (col == 0 ? 1.0 : 0.0) : monomial(P.monos + 3 * col, rel + 3 * (row - 1), d);
    }
    __syncwarp();
    // Householder QR, lane j owns columns j and j + 32
    for (int k = 0; k < M; ++k) {
      const double* vk = V + (size_t)k * LDW;
      if (lane == (k & 31)) {
        double s0 = 0, s1 = 0;
        int r = k;
        for (; r + 1 < m; r += 2) { s0 = fma(vk[r], vk[r], s0); s1 = fma(vk[r + 1], vk[r + 1], s1); }
        if (r < m) s0 = fma(vk[r], vk[r], s0);
        const double s = s0 + s1;
        const double x0 = vk[k];
        const double nr = sqrt(s);
        const double a = x0 >= 0 ? -nr : nr;
        const double vtv = 2.0 * (s - x0 * a);
        V[(size_t)k * LDW + k] = x0 - a;
        alpha[k] = a;
        beta[k] = vtv > 0 ? 2.0 / vtv : 0.0;
      }
      __syncwarp();
      const double bk = beta[k];
      for (int j = lane; j < M; j += 32) {
        if (j <= k) continue;
        double* vj = V + (size_t)j * LDW;
        double s0 = 0, s1 = 0;
        int r = k;
        for (; r + 1 < m; r += 2) { s0 = fma(vk[r], vj[r], s0); s1 = fma(vk[r + 1], vj[r + 1], s1); }
        if (r < m) s0 = fma(vk[r], vj[r], s0);
        const double sc = (s0 + s1) * bk;
        for (r = k; r < m; ++r) vj[r] = fma(-sc, vk[r], vj[r]);
      }
      __syncwarp();
    }
    bool ok;
    {
      double mx = 0, mn = 1e300;
      for (int k = lane; k < M; k += 32) { mx = fmax(mx, fabs(alpha[k])); mn = fmin(mn, fabs(alpha[k])); }
      for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      }
      ok = (mn >= 1e-8 * mx) && mx > 0;
    }
    if (!ok) continue;
    // stencil rows: quarter-warp t < nt solves for target t (ghost t < w, derivative t = w)
    const int nt = P.w + 1;                // ghosts and the normal derivative (every condition)
    const int t = lane >> 3, ql = lane & 7;
    double* y = Y + t * M;
    double* srow = S + t * LDW;
    if (t < nt) {
      if (t < P.w) {
        const int step = lo_sig ? 1 : -1;
        int mlo[3];
        {
          int64_t r = lo;
          mlo[0] = (int)(r % n); r /= n; mlo[1] = (int)(r % n); mlo[2] = d > 2 ? (int)(r / n) : 0;
        }
        int gm[3] = {mlo[0], mlo[1], mlo[2]};
        gm[ax] += (lo_sig ? 1 : 0) + t * step;
        double xi[3] = {0, 0, 0};
        for (int k = 0; k < d; ++k) xi[k] = (node_x(g, gm[k]) - xc[k]) / g.h;
        for (int col = ql; col < M; col += 8) y[col] = monomial(P.monos + 3 * col, xi, d);
      } else {
        for (int col = ql; col < M; col += 8) {
          const int* e = P.monos + 3 * col;
          double v = 0;
          if (e[0] + e[1] + e[2] == 1)
            for (int k = 0; k < d; ++k)
              if (e[k] == 1) v = nrm[k] / g.h;
          y[col] = v;
        }
      }
    }
    __syncwarp();
    for (int i = 0; i < M; ++i) {                       // y = R^-T c
      double part = 0;
      if (t < nt)
        for (int l = ql; l < i; l += 8) part = fma(V[(size_t)i * LDW + l], y[l], part);
      qw_sum(part);
      if (t < nt && ql == 0) y[i] = (y[i] - part) / alpha[i];
      __syncwarp();
    }
    if (t < nt)
      for (int r = ql; r < m; r += 8) srow[r] = r < M ? y[r] : 0.0;
    __syncwarp();
    for (int k = M - 1; k >= 0; --k) {                   // s = H_0 ... H_{M-1} [y; 0]
      const double* vk = V + (size_t)k * LDW;
      double dot = 0;
      if (t < nt)
        for (int r = k + ql; r < m; r += 8) dot = fma(vk[r], srow[r], dot);
      qw_sum(dot);
      dot *= beta[k];
      if (t < nt)
        for (int r = k + ql; r < m; r += 8) srow[r] = fma(-dot, vk[r], srow[r]);
      __syncwarp();
    }
    // outputs (same folding as the CTA kernel)
    const int rows = P.w + 1;
    double* coef = P.fit_coef + (size_t)f * rows * P.rcap;
    double* cdat = P.fit_cdat + (size_t)f * rows;
    if (P.bc == IIM_BC_NEUMANN) {
      double s2 = 0;
      for (int r = lane; r < m; r += 32) { const double v = P.beta_p * S[P.w * LDW + r]; s2 += v * v; }
      s2 = warp_sum(s2);
      const double Dc = P.beta_p * S[P.w * LDW];
      if (!(fabs(Dc) >= 1e-12 * sqrt(s2))) {
        if (lane == 0) set_status(P.status, IIM_ERR_SINGULAR);
        return;
      }
      for (int e = lane; e < P.w * R; e += 32) {
        const int k = e / R, al = e - k * R;
        coef[(size_t)k * P.rcap + al] = S[k * LDW + 1 + al] - S[k * LDW] * (P.beta_p * S[P.w * LDW + 1 + al]) / Dc;
      }
      if (lane < P.w) cdat[lane] = S[lane * LDW] / Dc;
      for (int e = lane; e < R; e += 32) coef[(size_t)P.w * P.rcap + e] = -(P.beta_p * S[P.w * LDW + 1 + e]) / Dc;
      if (lane == 0) cdat[P.w] = 1.0 / Dc;
    } else {
      for (int e = lane; e < nt * R; e += 32) {
        const int k = e / R, al = e - k * R;
        coef[(size_t)k * P.rcap + al] = S[k * LDW + 1 + al];
      }
      if (lane < nt) cdat[lane] = S[lane * LDW];
    }
    for (int e = lane; e < R; e += 32) P.fit_nodes[(size_t)f * P.rcap + e] = nodes[e];
    if (lane == 0) P.fit_R[f] = R;
    return;
  }
  if (lane == 0) overflow[f] = 2;       // the CTA kernel reports IIM_ERR_RANK if it fails as well
}

// 2D: a quarter-warp (8 lanes, rows over lanes) per fit and four fits per warp in
// lockstep, so that every FP64 instruction runs on all 32 lanes.  Only the first
// region size is tried here; fits that need a larger region, have too few or too
// many rows, or fail the rank test are flagged and redone by k_fit (one CTA each),
// which applies the same rules.
constexpr int kQuadRows = 48;          // rows of X_c a quarter-warp holds (q = 6: 38..46 rows; q = 4: about 23)

// Shared memory of one fit (doubles): V [M][LDQ], then the target rows S [4][LDQ] (which
// hold the node offsets [kQuadRows][2] before V is filled, and R^-T c_t in their first M
// entries before the reflectors are applied), alpha, 1/alpha, beta [M] each, and the node
// indices (ints).  LDQ is odd, so the eight lanes of a fit, each on its own column, hit
// distinct banks; the size is 8 mod 16 doubles, so the two fits of a half warp start 16
// banks apart.  M = 28: 13.5 KB per fit, four warps per SM.
struct QuadFitSmem {
  int M;
  __host__ __device__ int LDQ() const { return kQuadRows + 1; }
  __host__ __device__ size_t doubles() const {
    const int s_rel = 4 * LDQ() > 2 * kQuadRows ? 4 * LDQ() : 2 * kQuadRows;
    const size_t raw = (size_t)M * LDQ() + s_rel + 3 * M + kQuadRows / 2;
    return raw + ((8 - (int)(raw % 16)) + 16) % 16;
  }
};

__device__ inline void q8_sum(double& v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 2, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 1, 8);
}

template <int M>
__global__ void __launch_bounds__(32) k_fit_quad(FitParams P, QuadFitSmem Lq, int* __restrict__ overflow) {
  extern __shared__ double smq[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int qf = lane >> 3, ql = lane & 7;                   // fit slot in the warp, lane in the quarter
  const int f = (blockIdx.x * (blockDim.x >> 5) + wib) * 4 + qf;
  const GridView& g = P.g;
  const int nfit_here = P.interface_ ? 2 * (*P.K) : *P.K;
  const int LDQ = Lq.LDQ(), n = g.n;
  double* base = smq + (size_t)(wib * 4 + qf) * Lq.doubles();
  double* V = base;                      // [M][LDQ]
  double* S = V + (size_t)M * LDQ;       // [4][LDQ] (after the QR)
  double* rel = S;                       // [kQuadRows][2] (until V is filled)
  double* alpha = S + (4 * LDQ > 2 * kQuadRows ? 4 * LDQ : 2 * kQuadRows);   // [M]
  double* ialpha = alpha + M;            // [M]
  double* beta = ialpha + M;             // [M]
  int* nodes = (int*)(beta + M);         // [kQuadRows]
  bool active = f < nfit_here;
  const int c = P.interface_ ? (f >> 1) : f;
  const bool sig_plus = P.interface_ ? ((f & 1) == 0) : true;
  double xc[2] = {0, 0}, nrm[2] = {0, 0};
  int ax = 0;
  int64_t lo = 0;
  bool lo_sig = true;
  if (active) {
    xc[0] = P.cr_x[2 * c]; xc[1] = P.cr_x[2 * c + 1];
    nrm[0] = P.cr_n[2 * c]; nrm[1] = P.cr_n[2 * c + 1];
    ax = P.cr_axis[c];
    lo = P.cr_lo[c];
    lo_sig = (P.cr_loplus[c] != 0) == sig_plus;
  }
  const double ns0 = sig_plus ? -nrm[0] : nrm[0], ns1 = sig_plus ? -nrm[1] : nrm[1];
  const double an = P.q + 1.0, at = P.q / 2 + 1.0;
  const double an2 = an * an, at2 = at * at;
  const int rad = (int)ceil(an) + 1;
  int wlo0 = 0, wlo1 = 0, we0 = 1, we1 = 1;
  if (active) {
    const int c0 = (int)floor((xc[0] + 1.0) / g.h - 0.5), c1 = (int)floor((xc[1] + 1.0) / g.h - 0.5);
    wlo0 = max(0, c0 - rad); we0 = min(n, c0 + rad + 2) - wlo0;
    wlo1 = max(0, c1 - rad); we1 = min(n, c1 + rad + 2) - wlo1;
  }
  const int total = active ? we0 * we1 : 0;
  const double ih = 0.5 * n;                          // 1/h, exact
  // The phase-sigma node nearest to x_c is the sigma end of the cut edge: every other
  // node is at least h away while that end is t h <= h away (equality only when x_c
  // sits on the far node); that degenerate case takes the full search.
  int nearest;
  {
    const double tq = active ? P.cr_t[c] : 0.0;
    const double dnear = lo_sig ? tq : 1.0 - tq;      // distance to the sigma end, in h
    int anear = (int)lo;
    if (!lo_sig) anear += ax == 0 ? 1 : n;
    if (dnear < 1.0 - 1e-9) {
      nearest = anear;
    } else {
      double bd = 1e300;
      int bf = 0x7fffffff;
      for (int p = ql; p < total; p += 8) {
        const int i0 = wlo0 + p % we0, i1 = wlo1 + p / we0;
        const int fl = i0 + n * i1;
        if ((P.phase[fl] != 0) != sig_plus) continue;
        const double r0 = (node_x(g, i0) - xc[0]) * ih, r1 = (node_x(g, i1) - xc[1]) * ih;
        better(bd, bf, r0 * r0 + r1 * r1, fl);
      }
      for (int o = 4; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, bd, o, 8);
        const int of = __shfl_xor_sync(0xffffffffu, bf, o, 8);
        better(bd, bf, od, of);
      }
      nearest = bf;
    }
  }
  auto selected = [&](int p, int& fl, double& r0, double& r1) -> bool {
    const int i0 = wlo0 + p % we0, i1 = wlo1 + p / we0;
    fl = i0 + n * i1;
    if ((P.phase[fl] != 0) != sig_plus || fl == nearest) return false;
    r0 = (node_x(g, i0) - xc[0]) * ih;
    r1 = (node_x(g, i1) - xc[1]) * ih;
    const double d2 = r0 * r0 + r1 * r1, t = r0 * ns0 + r1 * ns1;
    const double tau2 = fmax(d2 - t * t, 0.0);
    // tau^2 / at^2 + t^2 / an^2 <= 1 multiplied through by at^2 an^2 (small exact integers)
    return t >= 0.0 && tau2 * an2 + (t * t) * at2 <= at2 * an2;
  };
  // one pass over the window: selection bits per lane (chunks of at most 64 positions)
  const int chunk = (total + 7) / 8;
  const int p0 = ql * chunk, p1 = min(total, p0 + chunk);
  unsigned long long bits = 0;
  int my = 0;
  for (int p = p0; p < p1 && p - p0 < 64; ++p) {
    int fl;
    double r0, r1;
    if (selected(p, fl, r0, r1)) { bits |= 1ull << (p - p0); ++my; }
  }
  int incl = my;
  for (int o = 1; o < 8; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o, 8);
    if (ql >= o) incl += y;
  }
  const int R = __shfl_sync(0xffffffffu, incl, 7, 8);
  if (active && (R > kQuadRows || R + 1 < M || chunk > 64)) {
    if (ql == 0) overflow[f] = 1;
    active = false;
  }
  if (active) {
    int o = incl - my;
    while (bits) {
      const int b = __ffsll((long long)bits) - 1;
      bits &= bits - 1;
      const int p = p0 + b;
      const int i0 = wlo0 + p % we0, i1 = wlo1 + p / we0;
      nodes[o] = i0 + n * i1;
      rel[2 * o] = (node_x(g, i0) - xc[0]) * ih;
      rel[2 * o + 1] = (node_x(g, i1) - xc[1]) * ih;
      ++o;
    }
  }
  __syncwarp();
  const int m = active ? R + 1 : 0;
  {
    // Vandermonde rows over the lanes: row 0 is x_c itself (xi = 0), row 1 + o the o-th
    // node.  Powers of each coordinate once per row, then one product per monomial, in
    // the graded order of the exponent table (degree, then decreasing x exponent).
    constexpr int Q = M == 28 ? 6 : 4;
    static_assert((Q + 1) * (Q + 2) / 2 == M, "2D monomial count");
    for (int row = ql; row < m; row += 8) {
      const double x0 = row == 0 ? 0.0 : rel[2 * (row - 1)], x1 = row == 0 ? 0.0 : rel[2 * (row - 1) + 1];
      double px[Q + 1], py[Q + 1];
      px[0] = 1.0;
      py[0] = 1.0;
#pragma unroll
      for (int e = 1; e <= Q; ++e) {
        px[e] = px[e - 1] * x0;
        py[e] = py[e - 1] * x1;
      }
      int col = 0;
#pragma unroll
      for (int deg = 0; deg <= Q; ++deg)
#pragma unroll
        for (int a = deg; a >= 0; --a) V[(size_t)(col++) * LDQ + row] = px[a] * py[deg - a];
    }
  }
  __syncwarp();
  // Householder QR.  The column's norm goes over the rows (8 lanes, tree sum); every lane
  // of the quarter forms the reflector's scalars, then each lane applies it to its own
  // trailing columns (k + 1 + ql, k + 9 + ql, ...): a product and an update over the rows
  // with no reduction across lanes.
  for (int k = 0; k < M; ++k) {
    double* vk = V + (size_t)k * LDQ;
    double s = 0;
    for (int r = k + ql; r < m; r += 8) s = fma(vk[r], vk[r], s);
    q8_sum(s);
    const double x0 = m > 0 ? vk[k] : 0.0;
    const double nr = sqrt(s);
    const double a = x0 >= 0 ? -nr : nr;
    const double vtv = 2.0 * (s - x0 * a);
    const double bk = vtv > 0 ? 2.0 / vtv : 0.0;
    __syncwarp();                       // vk[k] read by every lane before it changes
    if (ql == 0 && m > 0) {
      vk[k] = x0 - a;
      alpha[k] = a;
      beta[k] = bk;
    }
    __syncwarp();
    for (int j = k + 1 + ql; j < M; j += 8) {
      double* vj = V + (size_t)j * LDQ;
      double d0 = 0.0, d1 = 0.0;
      int r = k;
      for (; r + 1 < m; r += 2) {
        d0 = fma(vk[r], vj[r], d0);
        d1 = fma(vk[r + 1], vj[r + 1], d1);
      }
      if (r < m) d0 = fma(vk[r], vj[r], d0);
      const double sc = (d0 + d1) * bk;
      r = k;
      for (; r + 1 < m; r += 2) {
        vj[r] = fma(-sc, vk[r], vj[r]);
        vj[r + 1] = fma(-sc, vk[r + 1], vj[r + 1]);
      }
      if (r < m) vj[r] = fma(-sc, vk[r], vj[r]);
    }
    __syncwarp();
  }
  if (active) {
    double mx = 0, mn = 1e300;
    for (int k = 0; k < M; ++k) { mx = fmax(mx, fabs(alpha[k])); mn = fmin(mn, fabs(alpha[k])); }
    if (!(mn >= 1e-8 * mx && mx > 0)) {
      if (ql == 0) overflow[f] = 2;
      active = false;
    }
  }
  for (int k = ql; k < M; k += 8) ialpha[k] = active ? 1.0 / alpha[k] : 0.0;
  __syncwarp();
  // stencil rows of all targets together (rows over the 8 lanes)
  const int nt = P.w + 1;                // ghosts and the normal derivative (every condition)
  for (int t = 0; t < nt; ++t) {
    double* y = S + t * LDQ;
    if (t < P.w) {
      int mlo0 = (int)(lo % n), mlo1 = (int)(lo / n);
      int gm0 = mlo0, gm1 = mlo1;
      const int off = (lo_sig ? 1 : 0) + t * (lo_sig ? 1 : -1);
      if (ax == 0) gm0 += off; else gm1 += off;
      const double xi[2] = {(node_x(g, gm0) - xc[0]) * ih, (node_x(g, gm1) - xc[1]) * ih};
      for (int col = ql; col < M; col += 8) y[col] = monomial(P.monos + 3 * col, xi, 2);
    } else {
      for (int col = ql; col < M; col += 8) {
        const int* e = P.monos + 3 * col;
        y[col] = (e[0] + e[1] == 1) ? (e[0] ? nrm[0] : nrm[1]) * ih : 0.0;
      }
    }
  }
  __syncwarp();
  for (int i = 0; i < M; ++i) {                    // y_t = R^-T c_t, in place in S_t
    double part[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l = ql; l < i; l += 8) {
      const double rv = V[(size_t)i * LDQ + l];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < nt) part[t] = fma(rv, S[t * LDQ + l], part[t]);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (t < nt) q8_sum(part[t]);
    if (ql == 0)
      for (int t = 0; t < nt; ++t) S[t * LDQ + i] = (S[t * LDQ + i] - part[t]) * ialpha[i];
    __syncwarp();
  }
  for (int t = 0; t < nt; ++t)                      // [y_t; 0]
    for (int r = M + ql; r < m; r += 8) S[t * LDQ + r] = 0.0;
  __syncwarp();
  for (int k = M - 1; k >= 0; --k) {                // s_t = Q [y_t; 0]
    const double* vk = V + (size_t)k * LDQ;
    double d[4] = {0.0, 0.0, 0.0, 0.0};
    for (int r = k + ql; r < m; r += 8) {
      const double v = vk[r];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < nt) d[t] = fma(v, S[t * LDQ + r], d[t]);
    }
    const double bk = m > 0 ? beta[k] : 0.0;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (t < nt) {
        q8_sum(d[t]);
        d[t] *= bk;
      }
    for (int r = k + ql; r < m; r += 8) {
      const double v = vk[r];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < nt) S[t * LDQ + r] = fma(-d[t], v, S[t * LDQ + r]);
    }
    __syncwarp();
  }
  if (!active) return;
  const int rows = P.w + 1;
  double* coef = P.fit_coef + (size_t)f * rows * P.rcap;
  double* cdat = P.fit_cdat + (size_t)f * rows;
  if (P.bc == IIM_BC_NEUMANN) {
    double s2 = 0;
    for (int r = ql; r < m; r += 8) { const double v = P.beta_p * S[P.w * LDQ + r]; s2 += v * v; }
    // all lanes of this quarter are active here (the whole quarter shares `active`)
    s2 += __shfl_xor_sync(__activemask(), s2, 4, 8);
    s2 += __shfl_xor_sync(__activemask(), s2, 2, 8);
    s2 += __shfl_xor_sync(__activemask(), s2, 1, 8);
    const double Dc = P.beta_p * S[P.w * LDQ];
    if (!(fabs(Dc) >= 1e-12 * sqrt(s2))) {
      if (ql == 0) set_status(P.status, IIM_ERR_SINGULAR);
      return;
    }
    for (int e = ql; e < P.w * R; e += 8) {
      const int k = e / R, al = e - k * R;
      coef[(size_t)k * P.rcap + al] = S[k * LDQ + 1 + al] - S[k * LDQ] * (P.beta_p * S[P.w * LDQ + 1 + al]) / Dc;
    }
    if (ql < P.w) cdat[ql] = S[ql * LDQ] / Dc;
    for (int e = ql; e < R; e += 8) coef[(size_t)P.w * P.rcap + e] = -(P.beta_p * S[P.w * LDQ + 1 + e]) / Dc;
    if (ql == 0) cdat[P.w] = 1.0 / Dc;
  } else {
    for (int e = ql; e < nt * R; e += 8) {
      const int k = e / R, al = e - k * R;
      coef[(size_t)k * P.rcap + al] = S[k * LDQ + 1 + al];
    }
    if (ql < nt) cdat[ql] = S[ql * LDQ];
  }
  for (int e = ql; e < R; e += 8) P.fit_nodes[(size_t)f * P.rcap + e] = nodes[e];
  if (ql == 0) P.fit_R[f] = R;
}

// ------------------------------------------------------------------------------ Shortley-Weller levels
struct SWParams {
  GridView g;
  Geom G;
  int interface_, bc, box_bc;
  double beta_p, beta_m;
  // finest level only (else null): every cut edge is a control point whose root t is known
  const int32_t* edge_id;
  const double* cr_t;
  int cr_cap;
};

// side kinds
enum { S_REG = 0, S_DIR = 1, S_NEU = 2, S_IF = 3 };

__device__ inline void sw_side(const SWParams& P, const uint8_t* phase, int64_t i, const int* m, int ax, int s,
                               int& kind, double& psi, int* status) {
  const GridView& g = P.g;
  int pos = m[ax] + s;
  if (pos < 0 || pos >= g.n) {
    if (P.box_bc != IIM_BOX_DIRICHLET) set_status(status, IIM_ERR_GEOMETRY);
    kind = S_DIR;
    psi = 0.5;
    return;
  }
  int64_t nb = i + s * stride_of(g, ax);
  if (phase[nb] == phase[i]) { kind = S_REG; psi = 1.0; return; }
  if (P.interface_) { kind = S_IF; psi = 0.5; return; }
  int64_t lower = s > 0 ? i : nb;
  int ml[3];
  node_index(g, lower, ml);
  double t;
  const int c = P.cr_t ? P.edge_id[(int64_t)ax * g.N + lower] : -1;
  if (c >= 0 && c < P.cr_cap) {
    t = P.cr_t[c];                     // the same root k_crossings found on this edge
  } else {
    double x0[3] = {node_x(g, ml[0]), node_x(g, ml[1]), g.dim > 2 ? node_x(g, ml[2]) : 0.0};
    t = edge_root(P.G, x0, ax, g.h, g.dim);
  }
  double dist = s > 0 ? t : 1.0 - t;
  kind = P.bc == IIM_BC_DIRICHLET ? S_DIR : S_NEU;
  psi = fmax(dist, 0.5);               // intersections closer than h/2 are shifted (Sec. 3.1)
}

__global__ void k_sw_classify(SWParams P, const uint8_t* __restrict__ phase, int32_t* __restrict__ aux,
                              uint8_t* __restrict__ cls, int32_t* __restrict__ flag, int* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const GridView& g = P.g;
  if (i >= g.N) return;
  int f = 0;
  uint8_t c = phase[i] ? 4 : 0;        // phase +
  if (!(P.interface_ || phase[i])) {
    aux[i] = -2;
  } else {
    int m[3];
    node_index(g, i, m);
    for (int ax = 0; ax < g.dim; ++ax)
      for (int s = -1; s <= 1; s += 2) {
        int pos = m[ax] + s;
        if (pos < 0 || pos >= g.n || phase[i + s * stride_of(g, ax)] != phase[i]) f = 1;
      }
    aux[i] = -1;
    c |= f ? 3 : 1;                    // unknown, and irregular: its row is filled by k_sw_fill
  }
  cls[i] = c;
  flag[i] = f;
}

// one thread per irregular node (compacted), so that the FP64 root solves run on full warps
__global__ void k_sw_fill(SWParams P, const uint8_t* __restrict__ phase, const int32_t* __restrict__ list,
                          const int* __restrict__ count, int cap, int32_t* __restrict__ aux, double* tab64,
                          float* tab32, int* status) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const GridView& g = P.g;
  if (r >= *count || r >= cap) return;
  const int64_t i = list[r];
  int m[3];
  node_index(g, i, m);
  const int D = 2 * g.dim + 1;
  const double h2 = g.h * g.h;
  // interface wall weights (homogeneous Eq. 21, psi = 1/2): uw = lam_m u(minus node) + lam_p u(plus node)
  const double am = 0.5 / P.beta_m, ap = 0.5 / P.beta_p;
  const double lam_minus = ap / (ap + am), lam_plus = am / (ap + am);
  const bool self_plus = phase[i] != 0;
  const double lam_self = self_plus ? lam_plus : lam_minus, lam_other = self_plus ? lam_minus : lam_plus;
  double diag = 0, off[6];
  for (int ax = 0; ax < g.dim; ++ax) {
    int kl, kr;
    double pl, pr;
    sw_side(P, phase, i, m, ax, -1, kl, pl, status);
    sw_side(P, phase, i, m, ax, +1, kr, pr, status);
    bool nl = kl == S_NEU, nr = kr == S_NEU;
    double cl = 0, c0 = 0, cr = 0;
    if (!nl && !nr) {                       // Eq. 18 (Dirichlet form)
      cl = 2.0 / (pl * (pl + pr)) / h2;
      c0 = -2.0 / (pl * pr) / h2;
      cr = 2.0 / (pr * (pl + pr)) / h2;
    } else if (nl && !nr) {                 // Eq. 19a
      c0 = -2.0 / (pr * (2 * pl + pr)) / h2;
      cr = 2.0 / (pr * (2 * pl + pr)) / h2;
    } else if (nr && !nl) {                 // Eq. 19b (psi- in the denominators)
      cl = 2.0 / (pl * (pl + 2 * pr)) / h2;
      c0 = -2.0 / (pl * (pl + 2 * pr)) / h2;
    }
    diag += c0;
    double ol = 0, orr = 0;
    if (kl == S_REG) ol = cl;
    else if (kl == S_IF) { diag += cl * lam_self; ol = cl * lam_other; }
    if (kr == S_REG) orr = cr;
    else if (kr == S_IF) { diag += cr * lam_self; orr = cr * lam_other; }
    off[2 * ax] = ol;
    off[2 * ax + 1] = orr;
  }
  tab64[(size_t)r * D] = diag;
  tab32[(size_t)r * D] = (float)diag;
  for (int k = 0; k < 2 * g.dim; ++k) {
    tab64[(size_t)r * D + 1 + k] = off[k];
    tab32[(size_t)r * D + 1 + k] = (float)off[k];
  }
  aux[i] = r;
}

// outer-box sample points: face f = 2 ax + (side > 0), then the other node indices of the
// face in flat order (lowest remaining axis fastest); the point sits on the face
__global__ void k_box_points(GridView g, double* __restrict__ xb) {
  const int64_t per_face = g.N / g.n;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * g.dim * per_face) return;
  const int f = (int)(e / per_face), ax = f / 2;
  int64_t r = e - (int64_t)f * per_face;
  for (int k = 0; k < g.dim; ++k) {
    double v;
    if (k == ax) {
      v = (f & 1) ? 1.0 : -1.0;
    } else {
      const int m = (int)(r % g.n);
      r /= g.n;
      v = node_x(g, m);
    }
    xb[e * g.dim + k] = v;
  }
}

void box_points(Problem& P, double* xb, cudaStream_t s) {
  const int64_t B = 2 * P.g.dim * (P.g.N / P.g.n);
  IIM_LAUNCH(k_box_points, ceil_div(B, 256), 256, 0, s, P.g, xb);
}

// ------------------------------------------------------------------------------ host drivers
static Geom make_geom(const Problem& P) {
  const iim_problem_desc& d = P.desc;
  Geom G = {};
  G.kind = d.geom_kind;
  G.dim = d.dim;
  G.sign = d.plus_inside ? -1.0 : 1.0;
  for (int k = 0; k < 8; ++k) G.p[k] = d.geom_params[k];
  G.cs = std::cos(d.geom_params[4]);    // used by the ellipse only
  G.sn = std::sin(d.geom_params[4]);
  G.modes = (int)P.geom_coef.size() / 2;
  for (size_t k = 0; k < P.geom_coef.size() && k < 2 * kMaxFourierModes + 1; ++k) G.fc[k] = P.geom_coef[k];
  G.phi = P.phi_grid;
  G.gn = P.g.n;
  G.gh = P.g.h;
  return G;
}

iim_status setup_geometry(Problem& P, bool size_only) {
  cudaStream_t s = P.stream;
  P.geom = make_geom(P);
  const GridView& g = P.g;
  const int T = 256;
  IIM_LAUNCH(k_phase, ceil_div(g.N, T), T, 0, s, P.geom, g, P.phase);
  IIM_LAUNCH(k_edge_flags, ceil_div(g.N * g.dim, T), T, 0, s, g, P.phase, P.edge_flag);
  scan_exclusive(P.edge_flag, P.edge_id, g.N * g.dim, P.d_counts + 0, P.scan_scratch, s);
  if (size_only) return IIM_OK;
  IIM_LAUNCH(k_compact, ceil_div(g.N * g.dim, T), T, 0, s, P.edge_flag, P.edge_id, g.N * g.dim, P.K_cap, P.cr_edge,
             P.d_status);
  // one warp per block: the root solves are FP64-pipe bound (16 clocks per warp instruction
  // per SM), so a few thousand control points run fastest spread one warp per SM
  IIM_LAUNCH(k_crossings, ceil_div(P.K_cap, 32), 32, 0, s, P.geom, g, P.cr_edge, P.d_counts + 0, P.K_cap, P.phase,
             P.cr_axis, P.cr_lo, P.cr_loplus, P.cr_t, P.cr_x, P.cr_n, P.cr_kappa, P.d_status);
  IIM_LAUNCH(k_curvature_check, ceil_div(P.K_cap, T), T, 0, s, P.cr_kappa, P.d_counts + 0, g.h, P.d_status);
  WalkParams W{g, P.w, P.q, P.desc.bc == IIM_BC_INTERFACE, P.desc.box_bc};
  IIM_LAUNCH(k_affected_flags, ceil_div(g.N, T), T, 0, s, W, P.phase, P.aff_flag, P.d_status);
  scan_exclusive(P.aff_flag, P.aff_idx, g.N, P.d_counts + 1, P.scan_scratch, s);
  return IIM_OK;
}

iim_status setup_affected(Problem& P) {
  const int T = 256;
  WalkParams W{P.g, P.w, P.q, P.desc.bc == IIM_BC_INTERFACE, P.desc.box_bc};
  IIM_LAUNCH(k_affected_fill, ceil_div(P.g.N, T), T, 0, P.stream, W, P.phase, P.aff_flag, P.aff_idx, P.edge_id,
             P.aff_cap, P.aff_node, P.aff_fit, P.aff_j, P.d_status);
  return IIM_OK;
}

size_t fit_smem_bytes(const Problem& P) {
  size_t LD = P.rcap + 1;
  return sizeof(double) * ((size_t)P.M * LD + 4 * LD + 4 * P.M + 2 * P.M + 3 * (size_t)P.rcap) +
         sizeof(int) * (size_t)P.rcap;
}

iim_status setup_fits(Problem& P) {
  setup_affected(P);
  FitParams F;
  F.g = P.g;
  F.q = P.q;
  F.w = P.w;
  F.M = P.M;
  F.rcap = P.rcap;
  F.bc = P.desc.bc;
  F.interface_ = P.desc.bc == IIM_BC_INTERFACE;
  F.beta_p = P.desc.beta_plus;
  F.phase = P.phase;
  F.cr_axis = P.cr_axis;
  F.cr_lo = P.cr_lo;
  F.cr_loplus = P.cr_loplus;
  F.cr_t = P.cr_t;
  F.cr_x = P.cr_x;
  F.cr_n = P.cr_n;
  F.monos = P.d_monos;
  F.K = P.d_counts + 0;
  F.fit_R = P.fit_R;
  F.fit_nodes = P.fit_nodes;
  F.fit_coef = P.fit_coef;
  F.fit_cdat = P.fit_cdat;
  F.status = P.d_status;
  if (P.nfit_cap <= 0) return IIM_OK;
  // warp per fit
  WarpFitSmem W;
  W.M = P.M;
  W.RW = P.g.dim == 2 ? 64 : 128;
  W.LDW = W.RW + 1;
  const size_t per_warp = (W.bytes() / sizeof(double) + 1) * sizeof(double);
  int wpb = (int)((200 * 1024) / per_warp);
  wpb = wpb > 4 ? 4 : (wpb < 1 ? 1 : wpb);
  const size_t smw = per_warp * wpb;
  cudaError_t e = smem_optin((const void*)k_fit_warp);
  if (e != cudaSuccess) {
    set_error(std::string("least-squares kernel shared memory: ") + cudaGetErrorString(e));
    return IIM_ERR_CUDA;
  }
  cudaMemsetAsync(P.fit_overflow, 0, sizeof(int) * P.nfit_cap, P.stream);
  if (P.g.dim == 2 && (P.M == 15 || P.M == 28)) {
    QuadFitSmem Q;
    Q.M = P.M;
    const size_t smq = sizeof(double) * Q.doubles() * 4;       // one warp, four fits
    const void* kq = P.M == 15 ? (const void*)k_fit_quad<15> : (const void*)k_fit_quad<28>;
    e = smem_optin(kq);
    if (e != cudaSuccess) {
      set_error(std::string("least-squares kernel shared memory: ") + cudaGetErrorString(e));
      return IIM_ERR_CUDA;
    }
    if (P.M == 15) IIM_LAUNCH(k_fit_quad<15>, ceil_div(P.nfit_cap, 4), 32, smq, P.stream, F, Q, P.fit_overflow);
    else IIM_LAUNCH(k_fit_quad<28>, ceil_div(P.nfit_cap, 4), 32, smq, P.stream, F, Q, P.fit_overflow);
  } else {
    IIM_LAUNCH(k_fit_warp, ceil_div(P.nfit_cap, wpb), 32 * wpb, smw, P.stream, F, W, P.fit_overflow);
  }
  // CTA per fit for the flagged ones (more rows than a warp holds, or a grown region)
  size_t smem = fit_smem_bytes(P);
  if (smem > 48 * 1024) {
    e = smem_optin((const void*)k_fit);
    if (e != cudaSuccess) {
      set_error(std::string("least-squares kernel shared memory: ") + cudaGetErrorString(e));
      return IIM_ERR_CUDA;
    }
  }
  IIM_LAUNCH(k_fit, P.nfit_cap, kFitThreads, smem, P.stream, F, P.fit_overflow);
  return IIM_OK;
}

iim_status setup_levels(Problem& P, bool size_only) {
  const int T = 256;
  for (size_t l = 0; l < P.lv.size(); ++l) {
    Level& L = P.lv[l];
    SWParams S{L.g, P.geom, P.desc.bc == IIM_BC_INTERFACE, P.desc.bc, P.desc.box_bc, P.desc.beta_plus,
               P.desc.beta_minus, nullptr, nullptr, 0};
    if (l == 0 && !size_only && P.cr_t) {
      S.edge_id = P.edge_id;
      S.cr_t = P.cr_t;
      S.cr_cap = P.K_cap;
    }
    if (l > 0) IIM_LAUNCH(k_phase, ceil_div(L.g.N, T), T, 0, P.stream, P.geom, L.g, L.phase);
    IIM_LAUNCH(k_sw_classify, ceil_div(L.g.N, T), T, 0, P.stream, S, L.phase, L.aux, L.cls, L.flag, P.d_status);
    scan_exclusive(L.flag, L.idx, L.g.N, P.d_counts + 2 + (int)l, P.scan_scratch, P.stream);
    if (size_only) continue;
    IIM_LAUNCH(k_compact, ceil_div(L.g.N, T), T, 0, P.stream, L.flag, L.idx, L.g.N, L.irr_cap, L.irr_node,
               P.d_status);
    IIM_LAUNCH(k_sw_fill, ceil_div(L.irr_cap, 32), 32, 0, P.stream, S, L.phase, L.irr_node, P.d_counts + 2 + (int)l,
               L.irr_cap, L.aux, L.tab64, L.tab32, P.d_status);
  }
  return IIM_OK;
}

}  // namespace iim
