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
__global__ void __launch_bounds__(kFitThreads) k_fit(FitParams P) {
  extern __shared__ double sm[];
  const int f = blockIdx.x;
  const GridView& g = P.g;
  const int c = P.interface_ ? (f >> 1) : f;
  if (c >= *P.K) return;
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
    const int nt = (P.bc == IIM_BC_DIRICHLET) ? P.w : P.w + 1;
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

// ------------------------------------------------------------------------------ Shortley-Weller levels
struct SWParams {
  GridView g;
  Geom G;
  int interface_, bc, box_bc;
  double beta_p, beta_m;
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
  double x0[3] = {node_x(g, ml[0]), node_x(g, ml[1]), g.dim > 2 ? node_x(g, ml[2]) : 0.0};
  double t = edge_root(P.G, x0, ax, g.h, g.dim);
  double dist = s > 0 ? t : 1.0 - t;
  kind = P.bc == IIM_BC_DIRICHLET ? S_DIR : S_NEU;
  psi = fmax(dist, 0.5);               // intersections closer than h/2 are shifted (Sec. 3.1)
}

__global__ void k_sw_classify(SWParams P, const uint8_t* __restrict__ phase, int32_t* __restrict__ aux,
                              int32_t* __restrict__ flag, int* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const GridView& g = P.g;
  if (i >= g.N) return;
  int f = 0;
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
  }
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

// ------------------------------------------------------------------------------ host drivers
static Geom make_geom(const iim_problem_desc& d) {
  Geom G;
  G.kind = d.geom_kind;
  G.dim = d.dim;
  G.sign = d.plus_inside ? -1.0 : 1.0;
  for (int k = 0; k < 8; ++k) G.p[k] = d.geom_params[k];
  return G;
}

iim_status setup_geometry(Problem& P, bool size_only) {
  cudaStream_t s = P.stream;
  P.geom = make_geom(P.desc);
  const GridView& g = P.g;
  const int T = 256;
  IIM_LAUNCH(k_phase, ceil_div(g.N, T), T, 0, s, P.geom, g, P.phase);
  IIM_LAUNCH(k_edge_flags, ceil_div(g.N * g.dim, T), T, 0, s, g, P.phase, P.edge_flag);
  scan_exclusive(P.edge_flag, P.edge_id, g.N * g.dim, P.d_counts + 0, P.scan_scratch, s);
  if (size_only) return IIM_OK;
  IIM_LAUNCH(k_compact, ceil_div(g.N * g.dim, T), T, 0, s, P.edge_flag, P.edge_id, g.N * g.dim, P.K_cap, P.cr_edge,
             P.d_status);
  IIM_LAUNCH(k_crossings, ceil_div(P.K_cap, 128), 128, 0, s, P.geom, g, P.cr_edge, P.d_counts + 0, P.K_cap, P.phase,
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
  F.cr_x = P.cr_x;
  F.cr_n = P.cr_n;
  F.monos = P.d_monos;
  F.K = P.d_counts + 0;
  F.fit_R = P.fit_R;
  F.fit_nodes = P.fit_nodes;
  F.fit_coef = P.fit_coef;
  F.fit_cdat = P.fit_cdat;
  F.status = P.d_status;
  size_t smem = fit_smem_bytes(P);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_fit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
      set_error(std::string("least-squares kernel shared memory: ") + cudaGetErrorString(e));
      return IIM_ERR_CUDA;
    }
  }
  if (P.nfit_cap > 0) IIM_LAUNCH(k_fit, P.nfit_cap, kFitThreads, smem, P.stream, F);
  return IIM_OK;
}

iim_status setup_levels(Problem& P, bool size_only) {
  const int T = 256;
  for (size_t l = 0; l < P.lv.size(); ++l) {
    Level& L = P.lv[l];
    SWParams S{L.g, P.geom, P.desc.bc == IIM_BC_INTERFACE, P.desc.bc, P.desc.box_bc, P.desc.beta_plus,
               P.desc.beta_minus};
    if (l > 0) IIM_LAUNCH(k_phase, ceil_div(L.g.N, T), T, 0, P.stream, P.geom, L.g, L.phase);
    IIM_LAUNCH(k_sw_classify, ceil_div(L.g.N, T), T, 0, P.stream, S, L.phase, L.aux, L.flag, P.d_status);
    scan_exclusive(L.flag, L.idx, L.g.N, P.d_counts + 2 + (int)l, P.scan_scratch, P.stream);
    if (size_only) continue;
    IIM_LAUNCH(k_compact, ceil_div(L.g.N, T), T, 0, P.stream, L.flag, L.idx, L.g.N, L.irr_cap, L.irr_node,
               P.d_status);
    IIM_LAUNCH(k_sw_fill, ceil_div(L.irr_cap, 128), 128, 0, P.stream, S, L.phase, L.irr_node, P.d_counts + 2 + (int)l,
               L.irr_cap, L.aux, L.tab64, L.tab32, P.d_status);
  }
  return IIM_OK;
}

}  // namespace iim
