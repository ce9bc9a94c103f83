// Shared definitions of the GB300 IIM solver library (device code and host glue).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "../../include/iim.h"

namespace iim {

constexpr int kMaxDim = 3;
constexpr int kMaxW = 3;              // stencil half width (6th order)
constexpr int kMaxRestart = 16;       // FGMRES restart m
constexpr int kNumSMs = 152;

// status word bits written by device code (first error wins via atomicCAS)
__host__ __device__ inline int status_code(int s) { return s; }

// --------------------------------------------------------------------------- geometry
constexpr int kMaxFourierModes = 16;

struct Geom {
  int kind;
  int dim;
  double sign;                         // phi = sign * g
  double p[8];
  double cs, sn;                       // ellipse: cos and sin of the rotation angle p[4]
  int modes;                           // FOURIER: number of modes K
  double fc[2 * kMaxFourierModes + 1]; // FOURIER: a0, a1, b1, ..., aK, bK of r(theta)
  const double* phi;                   // LEVELSET_GRID: values at the n^dim nodes, x0 fastest
  int gn;                              // LEVELSET_GRID: nodes per axis
  double gh;                           // LEVELSET_GRID: node spacing 2 / gn
};

// ---------------------------------------------------------------------------------------
// Polar Fourier curve r(theta) = a0 + sum_k (a_k cos k theta + b_k sin k theta) around
// (p0, p1): r and its first two derivatives in theta.
__host__ __device__ inline void fourier_r(const Geom& G, double th, double* r, double* r1, double* r2) {
  double v = G.fc[0], d1 = 0, d2 = 0;
  for (int k = 1; k <= G.modes; ++k) {
    const double a = G.fc[2 * k - 1], b = G.fc[2 * k];
    double sk, ck;
    sincos(k * th, &sk, &ck);
    v += a * ck + b * sk;
    d1 += k * (b * ck - a * sk);
    d2 -= (double)k * k * (a * ck + b * sk);
  }
  *r = v;
  *r1 = d1;
  *r2 = d2;
}

// Level set given at the grid nodes: between nodes it is the tensor product of the degree-5
// Lagrange interpolants through the 6 nodes around the point along each axis (the stencil
// is shifted inwards at the grid's edge).  Along one axis, for coordinate x: s is the first
// stencil node and w0 / w1 / w2 the weights of the value and of its first and second
// derivative in x.  A coordinate equal to a node's (computed as for the grid) gets the
// weights of that node alone, so the interpolant takes the given values at the nodes.
__host__ __device__ inline void lag6(double x, int n, double h, int* s_out, double* w0, double* w1, double* w2) {
  const double tc = (x + 1.0) / h - 0.5;
  // A coordinate within 1e-9 h of node m counts as that node: the stencil starts at m - 2
  // and the local coordinate is the exact integer m - s, so the products below are exact,
  // the value weights are 1 and 0 and the interpolant returns the given value.  (The two
  // stencils that contain a node give it the same value but different derivatives, so the
  // choice must not depend on the last bit of the coordinate.)
  const int m = (int)floor(tc + 0.5);
  const bool at_node = fabs(tc - (double)m) <= 1e-9;
  int s = (at_node ? m : (int)floor(tc)) - 2;
  s = s < 0 ? 0 : (s > n - 6 ? n - 6 : s);
  *s_out = s;
  const double t = at_node ? (double)(m - s) : tc - (double)s;
  const double D[6] = {-120.0, 24.0, -12.0, 12.0, -24.0, 120.0};   // prod_{j != k} (k - j)
  double d[6];
  for (int k = 0; k < 6; ++k) d[k] = t - k;
  for (int k = 0; k < 6; ++k) {
    double v = 1.0;
    for (int j = 0; j < 6; ++j)
      if (j != k) v *= d[j];
    w0[k] = v / D[k];
    if (w1) {
      double a = 0.0;
      for (int j = 0; j < 6; ++j) {
        if (j == k) continue;
        double pr = 1.0;
        for (int l = 0; l < 6; ++l)
          if (l != k && l != j) pr *= d[l];
        a += pr;
      }
      w1[k] = a / (D[k] * h);
    }
    if (w2) {
      double a = 0.0;
      for (int j = 0; j < 6; ++j) {
        if (j == k) continue;
        for (int l = 0; l < 6; ++l) {
          if (l == k || l == j) continue;
          double pr = 1.0;
          for (int q = 0; q < 6; ++q)
            if (q != k && q != j && q != l) pr *= d[q];
          a += pr;
        }
      }
      w2[k] = a / (D[k] * h * h);
    }
  }
}

// value (der = -1), first derivative along axis der (0..dim-1), or second derivative
// d^2 / dx_a dx_b (der = 10 + 3 a + b) of the grid level set's interpolant at x
__host__ __device__ inline double levelset_eval(const Geom& G, const double* x, int der) {
  const int n = G.gn, d = G.dim;
  int s[3] = {0, 0, 0};
  double w[3][6];
  double t0[6], t1[6], t2[6];
  int da = -1, db = -1;
  if (der >= 10) { da = (der - 10) / 3; db = (der - 10) % 3; }
  else if (der >= 0) da = der;
  for (int ax = 0; ax < d; ++ax) {
    const int k1 = (ax == da) + (ax == db);        // derivative order along this axis
    lag6(x[ax], n, G.gh, &s[ax], t0, k1 >= 1 ? t1 : nullptr, k1 >= 2 ? t2 : nullptr);
    for (int k = 0; k < 6; ++k) w[ax][k] = k1 == 0 ? t0[k] : (k1 == 1 ? t1[k] : t2[k]);
  }
  double acc = 0.0;
  if (d == 2) {
    for (int j = 0; j < 6; ++j) {
      if (w[1][j] == 0.0) continue;
      const double* row = G.phi + (int64_t)(s[1] + j) * n + s[0];
      double r = 0.0;
      for (int i = 0; i < 6; ++i)
        if (w[0][i] != 0.0) r += w[0][i] * row[i];
      acc += w[1][j] * r;
    }
  } else {
    for (int l = 0; l < 6; ++l) {
      if (w[2][l] == 0.0) continue;
      double pl = 0.0;
      for (int j = 0; j < 6; ++j) {
        if (w[1][j] == 0.0) continue;
        const double* row = G.phi + ((int64_t)(s[2] + l) * n + (s[1] + j)) * n + s[0];
        double r = 0.0;
        for (int i = 0; i < 6; ++i)
          if (w[0][i] != 0.0) r += w[0][i] * row[i];
        pl += w[1][j] * r;
      }
      acc += w[2][l] * pl;
    }
  }
  return acc;
}

// Perturbed sphere: g = r - rho0 - rho1 c Q(d) / r^3 (-rho0 at the centre), d = x - centre, r = |d|,
// Q = (dx^2 - dy^2) dz, so that Q / r^3 is the degree-3 harmonic (e_x^2 - e_y^2) e_z of the
// direction e = d / r and c = 3 sqrt(3) / 2 scales its maximum on the sphere to 1.
constexpr double kPerturbScale = 2.598076211353316;

// g(x) < 0 inside the body; the paper's Omega+ = {phi >= 0}, phi = sign * g
__host__ __device__ inline double geom_g(const Geom& G, const double* x) {
  const double* p = G.p;
  switch (G.kind) {
    case IIM_GEOM_CIRCLE: return hypot(x[0] - p[0], x[1] - p[1]) - p[2];
    case IIM_GEOM_SPHERE: {
      double a = x[0] - p[0], b = x[1] - p[1], c = x[2] - p[2];
      return sqrt(a * a + b * b + c * c) - p[3];
    }
    case IIM_GEOM_ELLIPSE: {
      const double cs = G.cs, sn = G.sn;
      double dx = x[0] - p[0], dy = x[1] - p[1];
      double y0 = cs * dx + sn * dy, y1 = -sn * dx + cs * dy;
      return (y0 / p[2]) * (y0 / p[2]) + (y1 / p[3]) * (y1 / p[3]) - 1.0;
    }
    case IIM_GEOM_ELLIPSOID: {
      double a = (x[0] - p[0]) / p[3], b = (x[1] - p[1]) / p[4], c = (x[2] - p[2]) / p[5];
      return a * a + b * b + c * c - 1.0;
    }
    case IIM_GEOM_STAR: {
      double dx = x[0] - p[0], dy = x[1] - p[1];
      double rho = hypot(dx, dy), th = atan2(dy, dx);
      return rho - (p[2] + p[3] * sin(p[4] * th + p[5]));
    }
    case IIM_GEOM_FOURIER: {
      const double dx = x[0] - p[0], dy = x[1] - p[1];
      double r, r1, r2;
      fourier_r(G, atan2(dy, dx), &r, &r1, &r2);
      return hypot(dx, dy) - r;
    }
    case IIM_GEOM_LEVELSET_GRID: return levelset_eval(G, x, -1);
    case IIM_GEOM_PERTURBED_SPHERE: {
      double a = x[0] - p[0], b = x[1] - p[1], c = x[2] - p[2];
      double r = sqrt(a * a + b * b + c * c);
      if (r == 0.0) return -p[3];          // the centre: direction undefined, harmonic term 0
      return r - p[3] - p[4] * kPerturbScale * ((a * a - b * b) * c) / (r * r * r);
    }
  }
  return 0.0;
}

__host__ __device__ inline double geom_phi(const Geom& G, const double* x) { return G.sign * geom_g(G, x); }

__host__ __device__ inline void geom_grad_g(const Geom& G, const double* x, double* gr) {
  const double* p = G.p;
  switch (G.kind) {
    case IIM_GEOM_CIRCLE: {
      double a = x[0] - p[0], b = x[1] - p[1], r = hypot(a, b);
      gr[0] = a / r; gr[1] = b / r; return;
    }
    case IIM_GEOM_SPHERE: {
      double a = x[0] - p[0], b = x[1] - p[1], c = x[2] - p[2], r = sqrt(a * a + b * b + c * c);
      gr[0] = a / r; gr[1] = b / r; gr[2] = c / r; return;
    }
    case IIM_GEOM_ELLIPSE: {
      const double cs = G.cs, sn = G.sn;
      double dx = x[0] - p[0], dy = x[1] - p[1];
      double y0 = cs * dx + sn * dy, y1 = -sn * dx + cs * dy;
      double g0 = 2 * y0 / (p[2] * p[2]), g1 = 2 * y1 / (p[3] * p[3]);
      gr[0] = cs * g0 - sn * g1; gr[1] = sn * g0 + cs * g1; return;
    }
    case IIM_GEOM_ELLIPSOID: {
      gr[0] = 2 * (x[0] - p[0]) / (p[3] * p[3]);
      gr[1] = 2 * (x[1] - p[1]) / (p[4] * p[4]);
      gr[2] = 2 * (x[2] - p[2]) / (p[5] * p[5]);
      return;
    }
    case IIM_GEOM_STAR: {
      double dx = x[0] - p[0], dy = x[1] - p[1];
      double rho = hypot(dx, dy), th = atan2(dy, dx);
      double rp = p[3] * p[4] * cos(p[4] * th + p[5]);
      gr[0] = dx / rho + rp / rho * (dy / rho);
      gr[1] = dy / rho - rp / rho * (dx / rho);
      return;
    }
    case IIM_GEOM_FOURIER: {
      double dx = x[0] - p[0], dy = x[1] - p[1];
      double rho = hypot(dx, dy), r, rp, r2;
      fourier_r(G, atan2(dy, dx), &r, &rp, &r2);
      gr[0] = dx / rho + rp / rho * (dy / rho);
      gr[1] = dy / rho - rp / rho * (dx / rho);
      return;
    }
    case IIM_GEOM_LEVELSET_GRID: {
      for (int a = 0; a < G.dim; ++a) gr[a] = levelset_eval(G, x, a);
      return;
    }
    case IIM_GEOM_PERTURBED_SPHERE: {
      // grad g = d / r - rho1 c (grad Q r^-3 - 3 Q d r^-5)
      double d[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = sqrt(r2);
      double Q = (d[0] * d[0] - d[1] * d[1]) * d[2];
      double gQ[3] = {2 * d[0] * d[2], -2 * d[1] * d[2], d[0] * d[0] - d[1] * d[1]};
      double ir3 = 1.0 / (r2 * r), ir5 = ir3 / r2, k = p[4] * kPerturbScale;
      for (int i = 0; i < 3; ++i) gr[i] = d[i] / r - k * (gQ[i] * ir3 - 3 * Q * d[i] * ir5);
      return;
    }
  }
}

// Hessian of g (row major 3 x 3) for the perturbed sphere:
// (I - e e^T) / r - rho1 c [Hess Q r^-3 - 3 r^-5 (grad Q d^T + d grad Q^T) + Q (-3 r^-5 I + 15 r^-7 d d^T)]
__host__ __device__ inline void geom_hess_perturbed(const Geom& G, const double* x, double* H) {
  const double* p = G.p;
  double d[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
  double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], r = sqrt(r2);
  double Q = (d[0] * d[0] - d[1] * d[1]) * d[2];
  double gQ[3] = {2 * d[0] * d[2], -2 * d[1] * d[2], d[0] * d[0] - d[1] * d[1]};
  double HQ[9] = {2 * d[2], 0, 2 * d[0], 0, -2 * d[2], -2 * d[1], 2 * d[0], -2 * d[1], 0};
  double ir3 = 1.0 / (r2 * r), ir5 = ir3 / r2, ir7 = ir5 / r2, k = p[4] * kPerturbScale;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double del = i == j ? 1.0 : 0.0;
      const double hr = (del - d[i] * d[j] / r2) / r;
      const double hp = HQ[3 * i + j] * ir3 - 3 * (gQ[i] * d[j] + d[i] * gQ[j]) * ir5 +
                        Q * (-3 * del * ir5 + 15 * d[i] * d[j] * ir7);
      H[3 * i + j] = hr - k * hp;
    }
}

// largest |eigenvalue| of the shape operator P H P / |grad g| on the tangent plane of a
// 3D level surface (gr: grad g, H: Hessian of g, row major)
__host__ __device__ inline double shape_max_curvature3(const double* gr, const double* H) {
  double gn = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
  double n[3] = {gr[0] / gn, gr[1] / gn, gr[2] / gn};
  double a[3];
  if (fabs(n[0]) < 0.9) { a[0] = 1; a[1] = 0; a[2] = 0; } else { a[0] = 0; a[1] = 1; a[2] = 0; }
  double dt = a[0] * n[0] + a[1] * n[1] + a[2] * n[2];
  double t1[3] = {a[0] - dt * n[0], a[1] - dt * n[1], a[2] - dt * n[2]};
  double l = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
  t1[0] /= l; t1[1] /= l; t1[2] /= l;
  double t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
  double s11 = 0, s12 = 0, s22 = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      s11 += t1[i] * H[3 * i + j] * t1[j];
      s12 += t1[i] * H[3 * i + j] * t2[j];
      s22 += t2[i] * H[3 * i + j] * t2[j];
    }
  s11 /= gn; s12 /= gn; s22 /= gn;
  double m = 0.5 * (s11 + s22), dd = sqrt(0.25 * (s11 - s22) * (s11 - s22) + s12 * s12);
  return fmax(fabs(m + dd), fabs(m - dd));
}

// largest |principal curvature| of the level surface through x
__host__ __device__ inline double geom_curvature(const Geom& G, const double* x) {
  const double* p = G.p;
  switch (G.kind) {
    case IIM_GEOM_CIRCLE: return 1.0 / p[2];
    case IIM_GEOM_SPHERE: return 1.0 / p[3];
    case IIM_GEOM_STAR: {
      double th = atan2(x[1] - p[1], x[0] - p[0]);
      double s = sin(p[4] * th + p[5]), c = cos(p[4] * th + p[5]);
      double r = p[2] + p[3] * s, r1 = p[3] * p[4] * c, r2 = -p[3] * p[4] * p[4] * s;
      double den = r * r + r1 * r1;
      return fabs(r * r + 2 * r1 * r1 - r * r2) / (den * sqrt(den));
    }
    case IIM_GEOM_ELLIPSE: {
      // kappa = t^T H t / |grad g| for the unit tangent t
      double gr[2];
      geom_grad_g(G, x, gr);
      double gn = hypot(gr[0], gr[1]);
      double t0 = -gr[1] / gn, t1 = gr[0] / gn;
      const double cs = G.cs, sn = G.sn;
      double l0 = 2 / (p[2] * p[2]), l1 = 2 / (p[3] * p[3]);
      // H = R diag(l0,l1) R^T, R = [[cs,-sn],[sn,cs]]
      double u0 = cs * t0 + sn * t1, u1 = -sn * t0 + cs * t1;
      return fabs(l0 * u0 * u0 + l1 * u1 * u1) / gn;
    }
    case IIM_GEOM_ELLIPSOID: {
      double gr[3];
      geom_grad_g(G, x, gr);
      double gn = sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
      double n[3] = {gr[0] / gn, gr[1] / gn, gr[2] / gn};
      // orthonormal tangent basis
      double a[3];
      if (fabs(n[0]) < 0.9) { a[0] = 1; a[1] = 0; a[2] = 0; } else { a[0] = 0; a[1] = 1; a[2] = 0; }
      double d = a[0] * n[0] + a[1] * n[1] + a[2] * n[2];
      double t1[3] = {a[0] - d * n[0], a[1] - d * n[1], a[2] - d * n[2]};
      double l = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
      t1[0] /= l; t1[1] /= l; t1[2] /= l;
      double t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
      double H[3] = {2 / (p[3] * p[3]), 2 / (p[4] * p[4]), 2 / (p[5] * p[5])};
      double s11 = 0, s12 = 0, s22 = 0;
      for (int k = 0; k < 3; ++k) {
        s11 += H[k] * t1[k] * t1[k];
        s12 += H[k] * t1[k] * t2[k];
        s22 += H[k] * t2[k] * t2[k];
      }
      s11 /= gn; s12 /= gn; s22 /= gn;
      double m = 0.5 * (s11 + s22), dd = sqrt(0.25 * (s11 - s22) * (s11 - s22) + s12 * s12);
      return fmax(fabs(m + dd), fabs(m - dd));
    }
    case IIM_GEOM_FOURIER: {
      double r, r1, r2;
      fourier_r(G, atan2(x[1] - p[1], x[0] - p[0]), &r, &r1, &r2);
      double den = r * r + r1 * r1;
      return fabs(r * r + 2 * r1 * r1 - r * r2) / (den * sqrt(den));
    }
    case IIM_GEOM_LEVELSET_GRID: {
      double gr[3], H[9];
      for (int a = 0; a < G.dim; ++a) gr[a] = levelset_eval(G, x, a);
      for (int a = 0; a < G.dim; ++a)
        for (int b = a; b < G.dim; ++b) H[3 * a + b] = H[3 * b + a] = levelset_eval(G, x, 10 + 3 * a + b);
      if (G.dim == 2) {
        // curvature of the level curve: (g_xx g_y^2 - 2 g_xy g_x g_y + g_yy g_x^2) / |grad g|^3
        double gn = hypot(gr[0], gr[1]);
        return fabs(H[0] * gr[1] * gr[1] - 2 * H[1] * gr[0] * gr[1] + H[4] * gr[0] * gr[0]) / (gn * gn * gn);
      }
      return shape_max_curvature3(gr, H);
    }
    case IIM_GEOM_PERTURBED_SPHERE: {
      double gr[3], H[9];
      geom_grad_g(G, x, gr);
      geom_hess_perturbed(G, x, H);
      return shape_max_curvature3(gr, H);
    }
  }
  return 0.0;
}

// FP32 pre-check of the phase: returns +1 / -1 when the sign is certain, 0 otherwise
__device__ inline int geom_phase_fast(const Geom& G, const double* x) {
  if (G.kind != IIM_GEOM_STAR) return 0;
  float dx = (float)(x[0] - G.p[0]), dy = (float)(x[1] - G.p[1]);
  float rho = hypotf(dx, dy), th = atan2f(dy, dx);
  float g = rho - ((float)G.p[2] + (float)G.p[3] * sinf((float)G.p[4] * th + (float)G.p[5]));
  float margin = 1e-4f * (1.0f + (float)G.p[4]);
  if (g > margin) return G.sign > 0 ? 1 : -1;
  if (g < -margin) return G.sign > 0 ? -1 : 1;
  return 0;
}

__device__ inline bool phase_plus_at(const Geom& G, const double* x) {
  int f = geom_phase_fast(G, x);
  if (f != 0) return f > 0;
  return geom_phi(G, x) >= 0.0;
}

// Root of phi on the edge [x0, x0 + h e_ax]: safeguarded Newton with bisection.
// Returns t in [0,1] (fraction of h from x0).  Stops when the bracket or the
// Newton step is below 2 ulps of 1, i.e. at double precision.
__device__ inline double edge_root(const Geom& G, const double* x0, int ax, double h, int dim) {
  double x[3] = {x0[0], x0[1], dim > 2 ? x0[2] : 0.0};
  double lo = 0.0, hi = 1.0;
  bool s_lo = geom_phi(G, x) >= 0.0;
  double t = 0.5;
  for (int it = 0; it < 100; ++it) {
    x[ax] = x0[ax] + t * h;
    double f = geom_phi(G, x);
    if (f == 0.0) break;
    bool s = f >= 0.0;
    if (s == s_lo) lo = t; else hi = t;
    if (hi - lo <= 4.5e-16) break;
    double gr[3];
    geom_grad_g(G, x, gr);
    double df = G.sign * gr[ax] * h;
    double tn = (df != 0.0) ? t - f / df : 0.5 * (lo + hi);
    if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
    double step = fabs(tn - t);
    t = tn;
    if (step <= 4.5e-16) break;
  }
  return t < 0 ? 0 : (t > 1 ? 1 : t);
}

// --------------------------------------------------------------------------- small helpers
__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ inline float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline void set_status(int* st, int code) { atomicCAS(st, 0, code); }

// a restricted residual as stored: unchanged, or rounded to BF16 (round to nearest even)
__device__ inline float store_residual(float v, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}
__device__ inline double store_residual(double v, int) { return v; }

// The right-hand side f of a multigrid level as stored.  Levels whose f is a restricted
// residual in the BF16-residual form keep it as 2-byte BF16 values (rounded to nearest
// even when stored); every other f is stored in the level's precision.  Values read are
// those store_residual gives, so both forms of storage compute the same numbers.
__device__ inline float load_f(const float* f, int64_t i, int bf16) {
  return bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(f)[i]) : f[i];
}
__device__ inline double load_f(const double* f, int64_t i, int) { return f[i]; }
__device__ inline void store_f(float* f, int64_t i, float v, int bf16) {
  if (bf16) reinterpret_cast<__nv_bfloat16*>(f)[i] = __float2bfloat16_rn(v);
  else f[i] = v;
}
__device__ inline void store_f(double* f, int64_t i, double v, int) { f[i] = v; }
// two consecutive values (i even)
__device__ inline float2 load_f2(const float* f, int64_t i, int bf16) {
  if (bf16) return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(reinterpret_cast<const __nv_bfloat16*>(f) + i));
  return *reinterpret_cast<const float2*>(f + i);
}
__device__ inline double2 load_f2(const double* f, int64_t i, int) { return *reinterpret_cast<const double2*>(f + i); }

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Raise a kernel's dynamic shared memory limit to the most the device allows (beside the
// kernel's static shared memory), once per device and kernel.  The limit is a
// process-wide attribute of the function; setting it to each problem's own size would
// race with another thread launching the same kernel for a larger problem.
inline cudaError_t smem_optin(const void* func) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({dev, func})) return cudaSuccess;
  int mx = 0;
  cudaError_t e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.insert({dev, func});
  return e;
}

// launch accounting (every kernel launch of the library goes through IIM_LAUNCH)
void note_launch();
void note_launches(int64_t k);         // a graph launch that runs k kernels
#define IIM_LAUNCH(kernel, grid, block, smem, stream, ...)                \
  do {                                                                    \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);           \
    ::iim::note_launch();                                                 \
  } while (0)

// A launch that may begin before the previous kernel on the stream has finished
// (programmatic dependent launch): the kernel must run pdl_wait() before it reads anything
// the previous kernels write, and before it writes anything they read.  Used for the chain
// of multigrid level kernels, whose prologues read only set-up data.
#define IIM_LAUNCH_PDL(kernel_, grid_, block_, smem_, stream_, ...)                       \
  do {                                                                                     \
    cudaLaunchConfig_t cfg_ = {};                                                          \
    cfg_.gridDim = dim3(grid_);                                                            \
    cfg_.blockDim = dim3(block_);                                                          \
    cfg_.dynamicSmemBytes = (smem_);                                                       \
    cfg_.stream = (stream_);                                                               \
    cudaLaunchAttribute at_[1];                                                            \
    at_[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;                        \
    at_[0].val.programmaticStreamSerializationAllowed = 1;                                 \
    cfg_.attrs = at_;                                                                      \
    cfg_.numAttrs = 1;                                                                     \
    cudaLaunchKernelEx(&cfg_, kernel_, __VA_ARGS__);                                       \
    ::iim::note_launch();                                                                  \
  } while (0)

// wait until the kernels this one depends on have finished and their writes are visible
// (returns at once for a kernel launched without the programmatic attribute)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// let the next kernel on the stream start its prologue (it still waits for this one to finish)
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace iim
