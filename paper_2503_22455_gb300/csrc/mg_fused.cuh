// Fused Shortley-Weller multigrid kernels (paper Sec. 3.3), included by multigrid.cu.
//
// 2D fine levels: one CTA owns a TX x TY tile plus a halo of 3 (4 for the fused modes) in shared memory
// and runs several red/black half sweeps back to back on shrinking margins
// (temporal blocking), so each kernel reads and writes the level once:
//   MODE 0  first pre-smoothing sweep from u = 0; on the finest level the FP64
//           Krylov vector enters here: f = v * scale / beta_sigma
//   MODE 1  last pre-smoothing sweep, residual, 2x2 restriction to the coarse f
//   MODE 2  prolongation + correction, first post-smoothing sweep
//   MODE 3  last post-smoothing sweep; on the finest level z = (double) u
//   MODE 4  one plain sweep (only when nu > 2)
//   MODE 5  MODE 0 and MODE 1 in one kernel (nu1 = 2): halo 4, four half sweeps
//   MODE 6  MODE 2 and MODE 3 in one kernel (nu2 = 2)
//   MODE 7  MODE 5 from a given u (a W-cycle's second visit of a level): halo 5, since
//           the first half sweep now reads its neighbours
// Coarse tail: every level with at most 1024 nodes (one per thread) and the dense
// coarse solve run in a single CTA with the whole sub-hierarchy in shared memory.
#pragma once

namespace iim {

template <typename T>
struct LevelK {
  int dim, n;
  int64_t N;
  T ih2;          // 1/h^2
  T inv_dreg;     // 1/(-2d/h^2): inverse diagonal of a regular node
  T dreg;         // -2d/h^2
  const int32_t* aux;
  const T* tab;
  T* u;
  T* f;
  int f_bf16;     // f holds restricted residuals stored as BF16 (load_f / store_f)
};

template <typename T>
static LevelK<T> levk(const Level& L) {
  LevelK<T> k;
  k.dim = L.g.dim;
  k.n = L.g.n;
  k.N = L.g.N;
  const double h2 = L.g.h * L.g.h;
  k.ih2 = (T)(1.0 / h2);
  k.dreg = (T)(-2.0 * L.g.dim / h2);
  k.inv_dreg = (T)(-h2 / (2.0 * L.g.dim));
  k.aux = L.aux;
  k.tab = (const T*)(sizeof(T) == 8 ? (const void*)L.tab64 : (const void*)L.tab32);
  k.u = (T*)L.u;
  k.f = (T*)L.f;
  k.f_bf16 = L.f_bf16;
  return k;
}

constexpr int kH = 3;

// The point operations of the fine-level kernels, with every multiply-add fused explicitly
// and every other product kept unfused, so that the shared-memory tile kernels (here and
// in the batched engine) and the register-tiled ones give bit-identical results.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
// Gauss-Seidel value of a regular cell: (f - ih2 ((l + r) + (d + u))) / (-2d/h^2)
template <typename T>
__device__ __forceinline__ T gs_regular(T f, T s, T ih2, T inv_dreg) { return mul_rn(fma(-ih2, s, f), inv_dreg); }
// the off-diagonal sum of an irregular cell, c1 l + c2 r + c3 d + c4 u
template <typename T>
__device__ __forceinline__ T irr_offdiag(T c1, T c2, T c3, T c4, T l, T r, T d, T u) {
  return fma(c4, u, fma(c3, d, fma(c2, r, mul_rn(c1, l))));
}
// residual of a regular cell, f - (dreg u + ih2 s)
template <typename T>
__device__ __forceinline__ T res_regular(T f, T u, T s, T dreg, T ih2) { return f - fma(dreg, u, mul_rn(ih2, s)); }
// bilinear coarse-to-fine weights 9/16, 3/16, 3/16, 1/16
template <typename T>
__device__ __forceinline__ T prolong_bilinear(T e0, T e1, T e2, T e3) {
  return fma((T)0.0625, e3, fma((T)0.1875, e2, fma((T)0.1875, e1, mul_rn((T)0.5625, e0))));
}

template <typename T>
struct Fine2DParams {
  LevelK<T> L;
  LevelK<T> C;                 // coarse level (MODE 1, 2)
  const T* u_in;               // u is read from u_in (tile + halo) and written to u_out:
  T* u_out;                    // a kernel never reads what another CTA of it writes
  const T* uc;                 // MODE 2: the coarse correction
  int neumann;                 // Neumann prolongation: mean of the in-domain coarse neighbours
  const double* v;             // MODE 0 on the finest level: the Krylov vector
  const double* vscale;
  const uint8_t* phase;
  T inv_bp, inv_bm;
  double* z;                   // MODE 3 on the finest level: output
};

template <typename T>
__device__ inline T tab2(const LevelK<T>& L, int r, int k) { return L.tab[(size_t)r * 5 + k]; }

template <typename T, int TX, int TY, int MODE>
__device__ __forceinline__ void mg2d_tile(const Fine2DParams<T>& P, const int bx, const int by) {
  // the fused modes run four half sweeps on the tile; from a given u the first one needs
  // one more ring of neighbours
  constexpr int KH = MODE == 7 ? 5 : MODE >= 5 ? 4 : kH;
  constexpr bool DOWN_FIRST = MODE == 0 || MODE == 5, UP_FIRST = MODE == 2 || MODE == 6;
  constexpr bool UP_LAST = MODE == 3 || MODE == 6, RESTRICT = MODE == 1 || MODE == 5 || MODE == 7;
  constexpr int SX = TX + 2 * KH, SY = TY + 2 * KH, S = SX * SY;
  __shared__ T us[S];
  __shared__ T fs[S];
  __shared__ int as[S];
  // The irregular rows of the tile's cells, staged once: a cell with aux a >= 0 gets a slot
  // and as[e] = -3 - slot; past the capacity it keeps a and reads the level's table.
  constexpr int kIrrCap = sizeof(T) == 8 ? 96 : 256;
  __shared__ T ts[kIrrCap * 5];
  __shared__ int s_nirr;
  const LevelK<T>& L = P.L;
  const int n = L.n;
  const int x0 = bx * TX - KH, y0 = by * TY - KH;
  const bool finest_in = DOWN_FIRST && P.v != nullptr;
  const T vs = finest_in ? (T)(P.vscale ? *P.vscale : 1.0) : (T)1;
  const bool one_beta = P.inv_bp == P.inv_bm;       // no phase lookup for the scaling
  if (threadIdx.x == 0) s_nirr = 0;
  __syncthreads();
  {
    // all loads of a thread are issued before any is used (no aux -> f/u dependence)
    constexpr int NL = (S + 255) / 256;
    int ra[NL];
    T rf[NL], ru[NL];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + q * 256;
      const int sx = e % SX, sy = e / SX;
      const int gx = x0 + sx, gy = y0 + sy;
      ra[q] = -2;
      rf[q] = 0;
      ru[q] = 0;
      if (e < S && gx >= 0 && gx < n && gy >= 0 && gy < n) {
        const int64_t g = (int64_t)gy * n + gx;
        ra[q] = __ldg(L.aux + g);
        if (finest_in) rf[q] = mul_rn((T)__ldg(P.v + g), mul_rn(vs, one_beta || __ldg(P.phase + g) ? P.inv_bp : P.inv_bm));
        else rf[q] = load_f(L.f, g, L.f_bf16);
        if (!DOWN_FIRST) ru[q] = P.u_in[g];
      }
    }
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int e = threadIdx.x + q * 256;
      if (e >= S) continue;
      const bool unk = ra[q] != -2;
      us[e] = unk ? ru[q] : (T)0;
      fs[e] = unk ? rf[q] : (T)0;
      int a = ra[q];
      if (a >= 0) {
        const int slot = atomicAdd(&s_nirr, 1);
        if (slot < kIrrCap) {
#pragma unroll
          for (int k = 0; k < 5; ++k) ts[slot * 5 + k] = tab2(L, a, k);
          a = -3 - slot;
        }
      }
      as[e] = a;
    }
  }
  __syncthreads();
  // coefficient k of the irregular row of a cell (staged or from the level's table)
  auto cf = [&](int a, int k) -> T { return a <= -3 ? ts[(-3 - a) * 5 + k] : tab2(L, a, k); };
  if (finest_in) {
    // the finest level's right-hand side, stored before the residual replaces it in fs
    for (int e = threadIdx.x; e < TX * TY; e += blockDim.x) {
      const int tx = e % TX, ty = e / TX;
      const int gx = bx * TX + tx, gy = by * TY + ty;
      if (gx < n && gy < n) store_f(L.f, (int64_t)gy * n + gx, fs[(ty + KH) * SX + tx + KH], L.f_bf16);
    }
  }
  if (UP_FIRST) {
    // u += P e_coarse on margin 2 (4 when fused with the whole post-smoothing).  The coarse
    // u is 0 at coarse non-unknowns, so the bilinear form needs no aux; the Neumann mean
    // counts in-domain neighbours.
    const LevelK<T>& C = P.C;
    for (int e = threadIdx.x; e < S; e += blockDim.x) {
      const int sx = e % SX, sy = e / SX;
      constexpr int PM = MODE == 6 ? 4 : 2;
      if (sx < KH - PM || sx >= SX - (KH - PM) || sy < KH - PM || sy >= SY - (KH - PM)) continue;
      if (as[e] == -2) continue;
      const int gx = x0 + sx, gy = y0 + sy;
      const int I0 = gx >> 1, I1 = gy >> 1;
      const int s0 = (gx & 1) ? 1 : -1, s1 = (gy & 1) ? 1 : -1;
      T ev[4];
      int ok[4];
#pragma unroll
      for (int sel = 0; sel < 4; ++sel) {
        const int c0 = I0 + (sel & 1) * s0, c1 = I1 + (sel >> 1) * s1;
        ok[sel] = c0 >= 0 && c0 < C.n && c1 >= 0 && c1 < C.n;
        const int64_t ci = (int64_t)c1 * C.n + c0;
        ev[sel] = ok[sel] ? P.uc[ci] : (T)0;
        if (P.neumann) ok[sel] = ok[sel] && C.aux[ci] != -2;
      }
      T acc;
      if (P.neumann) {
        int cnt = ok[0] + ok[1] + ok[2] + ok[3];
        acc = cnt > 0 ? ((ok[0] ? ev[0] : 0) + (ok[1] ? ev[1] : 0) + (ok[2] ? ev[2] : 0) + (ok[3] ? ev[3] : 0)) / (T)cnt
                      : (T)0;
      } else {
        acc = prolong_bilinear(ev[0], ev[1], ev[2], ev[3]);
      }
      us[e] += acc;
    }
    __syncthreads();
  }
  auto half_sweep = [&](int colour, int margin, bool from_zero) {
    const int lo = KH - margin;
    const int rw = SX - 2 * lo, rh = SY - 2 * lo, hw = (rw + 1) / 2;
    for (int t = threadIdx.x; t < rh * hw; t += blockDim.x) {
      const int ry = t / hw, k2 = t - ry * hw;
      const int sy = lo + ry;
      // first x of this colour in the row: parity of (gx + gy) must equal colour
      const int par = ((x0 + lo + y0 + sy) & 1) != colour;
      const int sx = lo + 2 * k2 + par;
      if (sx >= SX - lo) continue;
      const int e = sy * SX + sx;
      const int a = as[e];
      if (a == -2) continue;
      T nv;
      if (a == -1) {
        const T s = from_zero ? (T)0 : (us[e - 1] + us[e + 1]) + (us[e - SX] + us[e + SX]);
        nv = gs_regular(fs[e], s, L.ih2, L.inv_dreg);
      } else {
        T s = 0;
        if (!from_zero)
          s = irr_offdiag(cf(a, 1), cf(a, 2), cf(a, 3), cf(a, 4), us[e - 1], us[e + 1], us[e - SX], us[e + SX]);
        const T dg = cf(a, 0);
        nv = dg != (T)0 ? (fs[e] - s) / dg : (T)0;
      }
      us[e] = nv;
    }
    __syncthreads();
  };
  if (MODE == 0) { half_sweep(0, 1, true); half_sweep(1, 0, false); }
  if (MODE == 1) { half_sweep(0, 2, false); half_sweep(1, 1, false); }
  if (MODE == 2 || MODE == 3 || MODE == 4) { half_sweep(0, 1, false); half_sweep(1, 0, false); }
  if (MODE == 5) {     // both pre-smoothing sweeps from u = 0
    half_sweep(0, 4, true); half_sweep(1, 3, false); half_sweep(0, 2, false); half_sweep(1, 1, false);
  }
  if (MODE == 6) {     // both post-smoothing sweeps after the correction
    half_sweep(0, 3, false); half_sweep(1, 2, false); half_sweep(0, 1, false); half_sweep(1, 0, false);
  }
  if (MODE == 7) {     // both pre-smoothing sweeps from u_in
    half_sweep(0, 4, false); half_sweep(1, 3, false); half_sweep(0, 2, false); half_sweep(1, 1, false);
  }
  if (RESTRICT) {
    // residual on the tile, kept in registers until every thread has read its neighbours
    constexpr int TPT = (TX * TY + 255) / 256;
    T rr[TPT];
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int e0 = threadIdx.x + q * 256;
      rr[q] = 0;
      if (e0 >= TX * TY) continue;
      const int tx = e0 % TX, ty = e0 / TX;
      const int e = (ty + KH) * SX + tx + KH;
      const int a = as[e];
      if (a == -1) {
        const T s = (us[e - 1] + us[e + 1]) + (us[e - SX] + us[e + SX]);
        rr[q] = res_regular(fs[e], us[e], s, L.dreg, L.ih2);
      } else if (a != -2) {
        const T s = irr_offdiag(cf(a, 1), cf(a, 2), cf(a, 3), cf(a, 4), us[e - 1], us[e + 1], us[e - SX], us[e + SX]);
        rr[q] = fs[e] - fma(cf(a, 0), us[e], s);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int e0 = threadIdx.x + q * 256;
      if (e0 >= TX * TY) continue;
      const int tx = e0 % TX, ty = e0 / TX;
      fs[(ty + KH) * SX + tx + KH] = rr[q];
    }
    __syncthreads();
    const LevelK<T>& C = P.C;
    for (int e = threadIdx.x; e < (TX / 2) * (TY / 2); e += blockDim.x) {
      const int cx = e % (TX / 2), cy = e / (TX / 2);
      const int gcx = bx * (TX / 2) + cx, gcy = by * (TY / 2) + cy;
      if (gcx >= C.n || gcy >= C.n) continue;
      const int64_t ci = (int64_t)gcy * C.n + gcx;
      const int b = (KH + 2 * cy) * SX + KH + 2 * cx;
      const T acc = (fs[b] + fs[b + 1]) + (fs[b + SX] + fs[b + SX + 1]);
      store_f(C.f, ci, C.aux[ci] == -2 ? (T)0 : acc * (T)0.25, C.f_bf16);
    }
  }
  for (int e = threadIdx.x; e < TX * TY; e += blockDim.x) {
    const int tx = e % TX, ty = e / TX;
    const int gx = bx * TX + tx, gy = by * TY + ty;
    if (gx >= n || gy >= n) continue;
    const int64_t g = (int64_t)gy * n + gx;
    const int se = (ty + KH) * SX + tx + KH;
    if (UP_LAST && P.z != nullptr) P.z[g] = (double)us[se];
    else P.u_out[g] = us[se];
  }
}

template <typename T, int TX, int TY, int MODE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 7 : 1) k_mg2d(Fine2DParams<T> P) {
  mg2d_tile<T, TX, TY, MODE>(P, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------- coarse tail (one CTA)
constexpr int kTailMaxLevels = 8;
constexpr int kTailNodes = 1024;      // levels with at most this many nodes go to the tail
constexpr int kTailThreads = 1024;    // threads of the tail's CTA: one node each on its first level

template <typename T>
struct TailParams {
  int nlev;                          // levels l0 .. l0+nlev-1; the last is the coarsest
  LevelK<T> L[kTailMaxLevels];
  int off[kTailMaxLevels + 1];       // offsets of the levels in the shared u / f / aux arrays
  int toff[kTailMaxLevels + 1];      // offsets (in T) of the levels' tables in shared memory
  const int* tcount[kTailMaxLevels]; // device counts of irregular rows per level
  int tcap[kTailMaxLevels];
  int stage_tables;                  // 1: tables copied to shared memory
  int nu1, nu2, neumann;
  int gamma;                         // visits of the next coarser level per visit (1: V, 2: W)
  int top_visits;                    // consecutive visits of the first level (gamma when the
                                     // tail is entered from a finer level, else 1)
  T* u_out;                          // where the first level's u goes (when z is not set)
  int ld;                            // stride of the coarse inverse (the coarsest level's nodes + aug)
  const int* nu_dev;                 // the coarsest level's unknowns (device count of the current set-up)
  int aug;                           // 1: the coarse system carries the augmentation (pure Neumann)
  const int32_t* map;                // node of each unknown of the coarse system (-1 past the unknowns)
  int* status;                       // where a coarse count out of range is reported
  const T* inv;                      // dense inverse of the coarsest SW matrix (row major)
  const double* v;                   // set when the tail starts at the finest level
  const double* vscale;
  const uint8_t* phase;
  T inv_bp, inv_bm;
  double* z;
};

template <typename T>
__device__ inline T tabd(const T* tb, int dim, int r, int k) { return tb[r * (2 * dim + 1) + k]; }

// offdiagonal part of (L u)_i from shared-memory u; m = (i0, i1, i2)
template <typename T, int DIM>
__device__ inline T tail_offdiag(const LevelK<T>& L, const T* tb, const T* u, int i, const int* m, int a) {
  const int n = L.n;
  if (a == -1) {
    T s = (u[i - 1] + u[i + 1]) + (u[i - n] + u[i + n]);
    if (DIM > 2) s += u[i - n * n] + u[i + n * n];
    return s * L.ih2;
  }
  T s = 0;
  int st = 1;
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    const T cl = tabd(tb, DIM, a, 1 + 2 * ax), cr = tabd(tb, DIM, a, 2 + 2 * ax);
    if (cl != (T)0 && m[ax] > 0) s += cl * u[i - st];
    if (cr != (T)0 && m[ax] < n - 1) s += cr * u[i + st];
    st *= n;
  }
  return s;
}

// node -> (i0, i1, i2) for the nodes i = t, t + stride, ...: one division per level, then
// a carry per step (stride is the block size)
template <int DIM>
struct NodeWalk {
  int n, i0, i1, i2, d0, drow;
  __device__ NodeWalk(int n_, int start, int stride) : n(n_) {
    i0 = start % n;
    const int r = start / n;
    i1 = DIM > 2 ? r % n : r;
    i2 = DIM > 2 ? r / n : 0;
    d0 = stride % n;
    drow = stride / n;
  }
  __device__ void advance() {
    i0 += d0;
    int rows = drow;
    if (i0 >= n) { i0 -= n; ++rows; }
    i1 += rows;
    if (DIM > 2 && i1 >= n) { i2 += i1 / n; i1 %= n; }
  }
};

template <typename T, int DIM>
__device__ __forceinline__ void vcycle_tail_body(const TailParams<T>& P, const double* v_in, const double* vscale,
                                                 double* z_out) {
  extern __shared__ unsigned char smraw[];
  const int tot = P.off[P.nlev];
  T* su = (T*)smraw;
  T* sf = su + tot;
  T* st = sf + tot;                                   // staged tables
  int* sa = (int*)(st + P.toff[P.nlev]);
  int* sco = sa + tot;                                 // node coordinates, i0 | i1 << 10 | i2 << 20
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k < P.nlev; ++k) {
    const int n = P.L[k].n;
    for (int i = tid; i < P.L[k].N; i += nt) {
      sa[P.off[k] + i] = P.L[k].aux[i];
      const int r = i / n;
      sco[P.off[k] + i] = (i - r * n) | ((DIM > 2 ? r % n : r) << 10) | ((DIM > 2 ? r / n : 0) << 20);
    }
  }
  if (P.stage_tables) {
    for (int k = 0; k < P.nlev; ++k) {
      const int rows = min(*P.tcount[k], P.tcap[k]);
      const int len = rows * (2 * DIM + 1);
      for (int e = tid; e < len; e += nt) st[P.toff[k] + e] = P.L[k].tab[e];
    }
  }
  auto table = [&](int k) -> const T* { return P.stage_tables ? st + P.toff[k] : P.L[k].tab; };
  // the staging above reads set-up data only; the right-hand side below is written by the
  // kernels before this one
  pdl_trigger();
  pdl_wait();
  {
    const LevelK<T>& L = P.L[0];
    const T vs = v_in ? (T)(vscale ? *vscale : 1.0) : (T)1;
    for (int i = tid; i < L.N; i += nt) {
      T f = 0;
      if (L.aux[i] != -2) f = v_in ? (T)v_in[i] * (vs * (P.phase[i] ? P.inv_bp : P.inv_bm)) : load_f(L.f, i, L.f_bf16);
      sf[i] = f;
    }
  }
  __syncthreads();
  // thread tid owns nodes tid, tid + blockDim.x, ... of every level (one node when N <= blockDim.x)
  auto sweep = [&](int k, int colour, bool from_zero) {
    const LevelK<T>& L = P.L[k];
    T* u = su + P.off[k];
    const T* f = sf + P.off[k];
    const T* tb = table(k);
    const int n = L.n;
    for (int i = tid; i < L.N; i += blockDim.x) {
      const int a = sa[P.off[k] + i];
      const int c = sco[P.off[k] + i];
      const int m[3] = {c & 1023, (c >> 10) & 1023, c >> 20};
      if (((m[0] + m[1] + m[2]) & 1) != colour) {
        if (from_zero) u[i] = 0;
      } else if (a == -2) {
        u[i] = 0;
      } else {
        const T s = from_zero ? (T)0 : tail_offdiag<T, DIM>(L, tb, u, i, m, a);
        if (a == -1) u[i] = (f[i] - s) * L.inv_dreg;
        else {
          const T dg = tabd(tb, DIM, a, 0);
          u[i] = dg != (T)0 ? (f[i] - s) / dg : (T)0;
        }
      }
    }
    __syncthreads();
  };
  // pre-smoothing of level k (the first sweep from u = 0 when zero) and the restriction
  // of its residual to level k + 1
  auto down = [&](int k, bool zero) {
    for (int it = 0; it < P.nu1; ++it) {
      sweep(k, 0, zero && it == 0);
      sweep(k, 1, false);
    }
    const LevelK<T>& L = P.L[k];
    const LevelK<T>& C = P.L[k + 1];
    const T* u = su + P.off[k];
    const T* f = sf + P.off[k];
    const int* aux = sa + P.off[k];
    const int* auxc = sa + P.off[k + 1];
    const T* tb = table(k);
    const T wch = DIM > 2 ? (T)0.125 : (T)0.25;
    NodeWalk<DIM> w(C.n, tid, nt);
    for (int I = tid; I < C.N; I += nt, w.advance()) {
      T acc = 0;
      if (auxc[I] != -2) {
        constexpr int nch = 1 << DIM;
        for (int c = 0; c < nch; ++c) {
          const int m[3] = {2 * w.i0 + (c & 1), 2 * w.i1 + ((c >> 1) & 1), DIM > 2 ? 2 * w.i2 + ((c >> 2) & 1) : 0};
          const int i = m[0] + L.n * (m[1] + L.n * m[2]);
          const int a = aux[i];
          if (a == -2) continue;
          const T dg = a == -1 ? L.dreg : tabd(tb, DIM, a, 0);
          acc += f[i] - (dg * u[i] + tail_offdiag<T, DIM>(L, tb, u, i, m, a));
        }
        acc *= wch;
      }
      sf[P.off[k + 1] + I] = store_residual(acc, C.f_bf16);
    }
    __syncthreads();
  };
  // the dense solve on the coarsest level (it does not depend on a starting u)
  auto coarse = [&]() {
    const int k = P.nlev - 1;
    const LevelK<T>& L = P.L[k];
    T* u = su + P.off[k];
    const T* f = sf + P.off[k];
    for (int i = tid; i < L.N; i += nt) u[i] = 0;
    __syncthreads();
    const int lane = tid & 31, wid = tid >> 5, nw = nt / 32;
    int nu = *P.nu_dev;                       // unknowns; the augmentation (if any) follows them
    if (nu < 0 || nu + P.aug > P.ld) {        // a count the dense system has no room for
      if (tid == 0 && P.status) set_status(P.status, IIM_ERR_CAPACITY);
      nu = 0;
    }
    for (int r = wid; r < nu; r += nw) {
      T s = 0;
      for (int c = lane; c < nu; c += 32) s += P.inv[(size_t)r * P.ld + c] * f[P.map[c]];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) u[P.map[r]] = s;
    }
    __syncthreads();
  };
  // level k += prolongated correction of level k + 1, then post-smoothing
  auto up = [&](int k) {
    const LevelK<T>& L = P.L[k];
    const LevelK<T>& C = P.L[k + 1];
    T* u = su + P.off[k];
    const T* ec = su + P.off[k + 1];
    const int* aux = sa + P.off[k];
    const int* auxc = sa + P.off[k + 1];
    NodeWalk<DIM> w(L.n, tid, nt);
    for (int i = tid; i < L.N; i += nt, w.advance()) {
      if (aux[i] == -2) continue;
      const int I[3] = {w.i0 >> 1, w.i1 >> 1, w.i2 >> 1};
      const int sg[3] = {(w.i0 & 1) ? 1 : -1, (w.i1 & 1) ? 1 : -1, (w.i2 & 1) ? 1 : -1};
      T acc = 0;
      int cnt = 0;
      constexpr int nsel = 1 << DIM;
      for (int sel = 0; sel < nsel; ++sel) {
        int c[3];
        T wgt = 1;
        bool inb = true;
        for (int q = 0; q < 3; ++q) {
          const int b = (sel >> q) & 1;
          c[q] = q < DIM ? I[q] + b * sg[q] : 0;
          if (q < DIM) {
            if (c[q] < 0 || c[q] >= C.n) inb = false;
            wgt *= b ? (T)0.25 : (T)0.75;
          }
        }
        if (!inb) continue;
        const int ci = c[0] + C.n * (c[1] + C.n * c[2]);
        if (auxc[ci] == -2) continue;
        if (P.neumann) { acc += ec[ci]; ++cnt; }
        else acc += wgt * ec[ci];
      }
      if (P.neumann) acc = cnt > 0 ? acc / (T)cnt : (T)0;
      u[i] += acc;
    }
    __syncthreads();
    for (int it = 0; it < P.nu2; ++it) {
      sweep(k, 0, false);
      sweep(k, 1, false);
    }
  };
  // Visit schedule (Sec. 3.3 results): each visit of level k below the first runs gamma
  // visits of level k + 1, the second from the first one's result with the same f; the
  // first level is visited top_visits times in a row.  Repeated coarsest visits within a
  // visit of the level above return the same u (the dense solve ignores the start), so
  // one is run.
  if (P.nlev == 1) {
    coarse();
  } else {
    int cnt[kTailMaxLevels];   // visits of level k + 1 completed in the current visit of level k
    int k = 0, top_done = 0;
    bool zero = true, descending = true;
    for (;;) {
      if (descending) {
        if (k == P.nlev - 1) {
          coarse();
          --k;
          cnt[k] = P.gamma;
          descending = false;
          continue;
        }
        down(k, zero);
        cnt[k] = 0;
        ++k;
        zero = true;
        continue;
      }
      if (cnt[k] < P.gamma) {       // another visit of level k + 1 from its current u
        ++k;
        zero = false;
        descending = true;
        continue;
      }
      up(k);
      if (k == 0) {
        if (++top_done < P.top_visits) {
          zero = false;
          descending = true;
          continue;
        }
        break;
      }
      --k;
      ++cnt[k];
    }
  }
  const LevelK<T>& L = P.L[0];
  for (int i = tid; i < L.N; i += nt) {
    const T u = su[i];
    if (z_out) z_out[i] = (double)u;
    else P.u_out[i] = u;
  }
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kTailThreads) k_vcycle_tail(TailParams<T> P) {
  vcycle_tail_body<T, DIM>(P, P.v, P.vscale, P.z);
}

}  // namespace iim
