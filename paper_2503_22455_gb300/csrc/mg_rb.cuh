// Red-black tile kernels for the fine levels of a 2D V(2,2) cycle (paper Sec. 3.3),
// included by multigrid.cu.
//
// The same two fused steps as MODE 5 and MODE 6 of mg_fused.cuh, with the same point
// operations in the same order (so every result is bit for bit the same), laid out so
// that a half sweep costs a handful of instructions per cell:
//   down  both pre-smoothing sweeps from u = 0, the residual and its 2x2 restriction
//         (on the finest level the FP64 Krylov vector enters here: f = v scale / beta)
//   up    the prolongated coarse correction, then both post-smoothing sweeps (on the
//         finest level the result leaves as the FP64 vector z)
//
// Layout.  A CTA owns a 64-column x SY-row window (the 56 x (SY - 8) output tile and a
// halo of 4).  The window starts at even grid coordinates, so cell (x, y) is red when
// x + y is even, and in row y the red cell of compressed column k sits at x = 2k + (y & 1),
// the black one at x = 2k + 1 - (y & 1).  Warp w owns rows w RW .. w RW + RW - 1 and lane k
// owns compressed column k of each, keeping the red and the black value of every one of its
// rows in registers.  A red cell's four neighbours are then black cells k + p - 1 and k + p
// of its row and k of the rows above and below (p = y & 1); a black cell's are red cells
// k - p and k + 1 - p and k above and below.  So of the horizontal pair one is the lane's own
// register and the other one shuffle away (lane k - 1 or k + 1), and the vertical pair is in
// the lane's own registers except at the warp's first and last rows, which each warp
// publishes in shared memory after every half sweep (one barrier per half sweep).  Outside
// the window (lanes -1 and 32, rows -1 and SY) the values are taken as zero: a cell at the
// window's edge computes a wrong value from them, and that error moves one cell inwards per
// half sweep, so after four half sweeps every cell at distance >= 3 (down) or >= 4 (up) from
// the edge is exact, which is what the residual and the output tile need.
//
// The restriction of a 2x2 block (two rows of one compressed column: one red and one black
// cell in each) is summed in registers by the lane that computed its four residuals.
// A cell's class is one byte (unknown, irregular row, phase +); irregular rows (cells
// next to the boundary or interface) take their five coefficients from the level's
// table, staged in shared memory; a warp takes that slower path only in the passes
// where one of its lanes has such a cell.
#pragma once

namespace iim {

constexpr int kRbKW = 32;                 // cells of one colour per window row
constexpr int kRbSX = 2 * kRbKW;          // window width
constexpr int kRbHalo = 4;
constexpr int kRbTX = kRbSX - 2 * kRbHalo;    // output columns per tile (56)
constexpr int kRbIrrCap = 320;            // staged irregular rows per tile

// cell classes (one byte per node and level)
constexpr uint8_t kClsUnknown = 1, kClsIrregular = 2, kClsPlus = 4;

template <typename T>
struct Rb2DParams {
  int n, nc;                 // fine and coarse level sizes
  T ih2, inv_dreg, dreg;
  const uint8_t* cls;        // fine level classes
  const int32_t* aux;        // table row of each irregular cell
  const T* tab;              // irregular rows: diag, left, right, down, up
  const T* f_in;             // the level's right-hand side (down on coarser levels; up)
  int f_bf16;                // f_in is stored as BF16
  T* f_out;                  // down on the finest level: f kept for the up step
  const double* v;           // down on the finest level: the Krylov vector
  const double* vscale;
  T inv_bp, inv_bm;
  const T* u_in;             // up: the level's u after the down step
  T* u_out;                  // down: the smoothed u; up on coarser levels: the result
  double* z;                 // up on the finest level: the result in FP64
  const T* uc;               // up: the coarse correction
  const uint8_t* cls_c;      // coarse classes
  T* fc;                     // down: the coarse right-hand side
  int fc_bf16;
  int neumann;
};

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// shared-memory bytes of one CTA of the kernel below
template <typename T, int NW, int RW, bool UP>
constexpr size_t rb_smem_bytes() {
  return sizeof(T) * 2 * (size_t)NW * 2 * 32                    // published first / last rows
         + sizeof(T) * 5 * (size_t)kRbIrrCap                    // staged irregular rows
         + sizeof(int) * (size_t)kRbIrrCap                      // their nodes
         + sizeof(int16_t) * (size_t)NW * RW * kRbSX            // slot of each irregular cell
         + (UP ? (sizeof(T) + 1) * (size_t)(NW * RW / 2 + 2) * (kRbKW + 2) : 0)   // coarse window
         + 16;
}

template <typename T, int NW, int RW, bool UP>
// two-row windows fit in 40 registers (no spills): 1536 threads per SM; four-row windows would spill there
__global__ void __launch_bounds__(NW * 32, RW == 2 ? 1536 / (NW * 32) : 1024 / (NW * 32)) k_mg2d_rb(Rb2DParams<T> P) {
  constexpr int SY = NW * RW, TY = SY - 2 * kRbHalo;
  static_assert(RW % 2 == 0, "a lane's rows come in pairs (the 2x2 restriction)");
  static_assert(SY > 2 * kRbHalo, "the window must be taller than its two halos");
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char rb_smem[];
  T* sPub = (T*)rb_smem;                                   // [colour][warp][first, last][lane]
  T* sTab = sPub + 2 * NW * 2 * 32;
  int* sList = (int*)(sTab + 5 * kRbIrrCap);
  int16_t* sCode = (int16_t*)(sList + kRbIrrCap);
  T* sUc = (T*)(sCode + SY * kRbSX);                       // up: coarse window (SY/2 + 2) x 34
  uint8_t* sOk = (uint8_t*)(sUc + (SY / 2 + 2) * (kRbKW + 2));
  __shared__ int s_nirr;

  const uint8_t* __restrict__ cls = P.cls;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n = P.n;
  const int x0 = blockIdx.x * kRbTX - kRbHalo, y0 = blockIdx.y * TY - kRbHalo;
  const bool finest_in = !UP && P.v != nullptr;
  const bool one_beta = P.inv_bp == P.inv_bm;
  auto in_tile = [&](int y) { return y >= kRbHalo && y < SY - kRbHalo && lane >= kRbHalo / 2 && lane < kRbKW - kRbHalo / 2; };

  if (threadIdx.x == 0) s_nirr = 0;

  // ---------------------------------------------------------------- load
  // Set-up data first (class codes, irregular rows and their table entries): this runs while
  // the previous level kernel may still be finishing.  Then the data the previous kernels
  // write (right-hand side, u), after pdl_wait().
  const int gx = x0 + 2 * lane;
  uchar2 cc[RW];
#pragma unroll
  for (int j = 0; j < RW; ++j) {
    const int gy = y0 + warp * RW + j;
    const bool in = gy >= 0 && gy < n && gx >= 0 && gx < n;    // n even: gx + 1 < n too
    cc[j] = in ? __ldg((const uchar2*)(cls + (int64_t)gy * n + gx)) : make_uchar2(0, 0);
  }
  unsigned unk = 0, irr = 0;          // bit 2 j + c: cell of row j, colour c (0 red, 1 black)
#pragma unroll
  for (int j = 0; j < RW; ++j) {
    const int p = j & 1;
    // x = 2 lane is red when p = 0
    const uint8_t cr = p ? cc[j].y : cc[j].x, cb = p ? cc[j].x : cc[j].y;
    unk |= ((cr & kClsUnknown) ? 1u : 0u) << (2 * j);
    unk |= ((cb & kClsUnknown) ? 1u : 0u) << (2 * j + 1);
    irr |= ((cr & kClsIrregular) ? 1u : 0u) << (2 * j);
    irr |= ((cb & kClsIrregular) ? 1u : 0u) << (2 * j + 1);
  }
  __syncthreads();                    // s_nirr
  // irregular cells: a slot each (code < 0: past the staging capacity, read from the table)
#pragma unroll
  for (int j = 0; j < RW; ++j) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      if (!((irr >> (2 * j + c)) & 1u)) continue;
      const int y = warp * RW + j, p = j & 1;
      const int x = 2 * lane + (c == 0 ? p : 1 - p);
      const int slot = atomicAdd(&s_nirr, 1);
      if (slot < kRbIrrCap) sList[slot] = (y0 + y) * n + (x0 + x);
      sCode[y * kRbSX + x] = (int16_t)(slot < kRbIrrCap ? slot : -1);
    }
  }
  // which passes (row j, colour c) have an irregular cell in this warp
  const unsigned irr_w = __reduce_or_sync(0xffffffffu, irr);
  __syncthreads();
  {
    // the staged rows, loaded by the whole CTA (two dependent loads per row, all rows at once)
    const int nirr = min(s_nirr, kRbIrrCap);
    for (int r = threadIdx.x; r < nirr; r += NW * 32) {
      const int a = __ldg(P.aux + sList[r]);
#pragma unroll
      for (int k = 0; k < 5; ++k) sTab[r * 5 + k] = P.tab[(size_t)a * 5 + k];
    }
  }
  pdl_trigger();
  pdl_wait();
  // every load of the lane's right-hand side and u is issued before any of them is used
  T f0[RW], f1[RW], u0[RW], u1[RW];
#pragma unroll
  for (int j = 0; j < RW; ++j) {
    const int gy = y0 + warp * RW + j;
    const bool in = gy >= 0 && gy < n && gx >= 0 && gx < n;
    const int64_t g = (int64_t)gy * n + gx;
    f0[j] = f1[j] = u0[j] = u1[j] = (T)0;
    if (in) {
      if (finest_in) {
        const double2 vv = __ldg((const double2*)(P.v + g));
        f0[j] = (T)vv.x;
        f1[j] = (T)vv.y;
      } else {
        const T2 ff = load_f2(P.f_in, g, P.f_bf16);
        f0[j] = ff.x;
        f1[j] = ff.y;
      }
      if (UP) {
        const T2 uu = *(const T2*)(P.u_in + g);
        u0[j] = uu.x;
        u1[j] = uu.y;
      }
    }
  }
  const T vs = finest_in ? (T)(P.vscale ? *P.vscale : 1.0) : (T)1;
  T fr[RW], fb[RW], ur[RW], ub[RW];
#pragma unroll
  for (int j = 0; j < RW; ++j) {
    const int y = warp * RW + j, p = j & 1;
    const uint8_t c0 = cc[j].x, c1 = cc[j].y;
    T a0 = f0[j], a1 = f1[j];
    if (finest_in) {
      a0 = mul_rn(a0, mul_rn(vs, one_beta || (c0 & kClsPlus) ? P.inv_bp : P.inv_bm));
      a1 = mul_rn(a1, mul_rn(vs, one_beta || (c1 & kClsPlus) ? P.inv_bp : P.inv_bm));
    }
    T b0 = u0[j], b1 = u1[j];
    if (!(c0 & kClsUnknown)) a0 = b0 = 0;
    if (!(c1 & kClsUnknown)) a1 = b1 = 0;
    fr[j] = p ? a1 : a0;
    fb[j] = p ? a0 : a1;
    ur[j] = p ? b1 : b0;
    ub[j] = p ? b0 : b1;
    if (finest_in && in_tile(y) && y0 + y < n && gx < n) {
      // the finest level's right-hand side, for the up step
      T2 st;
      st.x = a0;
      st.y = a1;
      *(T2*)(P.f_out + (int64_t)(y0 + y) * n + gx) = st;
    }
  }
  auto coef_of = [&](int j, int c, T* cf) {
    const int y = warp * RW + j, p = j & 1;
    const int x = 2 * lane + (c == 0 ? p : 1 - p);
    const int code = sCode[y * kRbSX + x];
    if (code >= 0) {
#pragma unroll
      for (int k = 0; k < 5; ++k) cf[k] = sTab[code * 5 + k];
    } else {
      const int a = P.aux[(int64_t)(y0 + y) * n + (x0 + x)];
#pragma unroll
      for (int k = 0; k < 5; ++k) cf[k] = P.tab[(size_t)a * 5 + k];
    }
  };

  if (UP) {
    // coarse window: coarse nodes x0/2 - 1 .. x0/2 + 32, y0/2 - 1 .. y0/2 + SY/2
    constexpr int CW = kRbKW + 2, CH = SY / 2 + 2;
    const int cx0 = x0 / 2 - 1, cy0 = y0 / 2 - 1, nc = P.nc;
    for (int e = threadIdx.x; e < CW * CH; e += NW * 32) {
      const int r = e / CW, k = e - r * CW;
      const int cx = cx0 + k, cy = cy0 + r;
      T val = 0;
      uint8_t ok = 0;
      if (cx >= 0 && cx < nc && cy >= 0 && cy < nc) {
        const int64_t ci = (int64_t)cy * nc + cx;
        val = P.uc[ci];
        ok = P.neumann ? (P.cls_c[ci] & kClsUnknown) : 1;
      }
      sUc[e] = val;
      sOk[e] = ok;
    }
    __syncthreads();
    // u += P e_coarse at every unknown of the window
#pragma unroll
    for (int j = 0; j < RW; ++j) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        if (!((unk >> (2 * j + c)) & 1u)) continue;
        const int y = warp * RW + j, p = j & 1;
        const int x = 2 * lane + (c == 0 ? p : 1 - p);
        // window-relative coarse parent (gx >> 1 with x0 even) and the side of each axis
        const int I0 = (x >> 1) + 1, I1 = (y >> 1) + 1;
        const int s0 = (x & 1) ? 1 : -1, s1 = (y & 1) ? 1 : -1;
        T ev[4];
        int ok[4];
#pragma unroll
        for (int sel = 0; sel < 4; ++sel) {
          const int e = (I1 + (sel >> 1) * s1) * CW + I0 + (sel & 1) * s0;
          ev[sel] = sUc[e];
          ok[sel] = sOk[e];
        }
        T acc;
        if (P.neumann) {
          const int cnt = ok[0] + ok[1] + ok[2] + ok[3];
          acc = cnt > 0 ? ((ok[0] ? ev[0] : 0) + (ok[1] ? ev[1] : 0) + (ok[2] ? ev[2] : 0) + (ok[3] ? ev[3] : 0)) /
                              (T)cnt
                        : (T)0;
        } else {
          acc = prolong_bilinear(ev[0], ev[1], ev[2], ev[3]);
        }
        if (c == 0) ur[j] += acc;
        else ub[j] += acc;
      }
    }
  }
  // the warp's first and last rows, for the vertical neighbours of the warps around it
  auto pub = [&](int c, int w, int which) -> T* { return sPub + ((c * NW + w) * 2 + which) * 32; };
  auto publish = [&](int c) {
    pub(c, warp, 0)[lane] = c == 0 ? ur[0] : ub[0];
    pub(c, warp, 1)[lane] = c == 0 ? ur[RW - 1] : ub[RW - 1];
  };
  // the four neighbours (values of the other colour) of the colour-c cell of row j
  auto nbrs = [&](int j, int c, T& lft, T& rgt, T& dn, T& upv) {
    const int p = j & 1;
    const T own = c == 0 ? ub[j] : ur[j];            // other colour, same compressed column
    if ((c == 0) == (p == 0)) {                      // red p = 0, black p = 1: left from lane - 1
      const T v = __shfl_up_sync(0xffffffffu, own, 1);
      lft = lane == 0 ? (T)0 : v;
      rgt = own;
    } else {                                         // red p = 1, black p = 0: right from lane + 1
      const T v = __shfl_down_sync(0xffffffffu, own, 1);
      lft = own;
      rgt = lane == 31 ? (T)0 : v;
    }
    if (j > 0) dn = c == 0 ? ub[j - 1] : ur[j - 1];
    else dn = warp > 0 ? pub(1 - c, warp - 1, 1)[lane] : (T)0;
    if (j < RW - 1) upv = c == 0 ? ub[j + 1] : ur[j + 1];
    else upv = warp < NW - 1 ? pub(1 - c, warp + 1, 0)[lane] : (T)0;
  };
  publish(0);
  publish(1);
  __syncthreads();

  // ---------------------------------------------------------------- four half sweeps
  auto half_sweep = [&](const int colour, const bool from_zero) {
#pragma unroll
    for (int j = 0; j < RW; ++j) {
      const int bit = 2 * j + colour;
      const T f = colour == 0 ? fr[j] : fb[j];
      T lft = 0, rgt = 0, dn = 0, upv = 0;
      if (!from_zero) nbrs(j, colour, lft, rgt, dn, upv);
      T nv = gs_regular(f, from_zero ? (T)0 : (lft + rgt) + (dn + upv), P.ih2, P.inv_dreg);
      if ((irr_w >> bit) & 1u) {
        if ((irr >> bit) & 1u) {
          T cf[5];
          coef_of(j, colour, cf);
          T s = 0;
          if (!from_zero) s = irr_offdiag(cf[1], cf[2], cf[3], cf[4], lft, rgt, dn, upv);
          nv = cf[0] != (T)0 ? (f - s) / cf[0] : (T)0;
        }
      }
      if ((unk >> bit) & 1u) {
        if (colour == 0) ur[j] = nv;
        else ub[j] = nv;
      }
    }
    publish(colour);
    __syncthreads();
  };
  half_sweep(0, !UP);
  half_sweep(1, false);
  half_sweep(0, false);
  half_sweep(1, false);

  if (!UP) {
    // ---------------------------------------------------------------- residual, restriction
    const int nc = P.nc;
#pragma unroll
    for (int j = 0; j < RW; j += 2) {
      const int y = warp * RW + j;        // even: rows y, y + 1 form the 2x2 blocks
      if (y < kRbHalo || y >= SY - kRbHalo) continue;          // warp-uniform
      T r[2][2];                            // [row j, j + 1][red, black]
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int bit = 2 * (j + jj) + c;
          T lft, rgt, dn, upv;
          nbrs(j + jj, c, lft, rgt, dn, upv);
          const T u = c == 0 ? ur[j + jj] : ub[j + jj];
          const T f = c == 0 ? fr[j + jj] : fb[j + jj];
          T rr = 0;
          if ((unk >> bit) & 1u) {
            if ((irr >> bit) & 1u) {
              T cf[5];
              coef_of(j + jj, c, cf);
              const T s = irr_offdiag(cf[1], cf[2], cf[3], cf[4], lft, rgt, dn, upv);
              rr = f - fma(cf[0], u, s);
            } else {
              rr = res_regular(f, u, (lft + rgt) + (dn + upv), P.dreg, P.ih2);
            }
          }
          r[jj][c] = rr;
        }
      }
      // x order in the block: row y (p = 0) red then black, row y + 1 (p = 1) black then red
      const int gcx = (x0 + kRbHalo) / 2 + lane - kRbHalo / 2;
      const int gcy = (y0 + kRbHalo) / 2 + (y - kRbHalo) / 2;
      if (lane >= kRbHalo / 2 && lane < kRbKW - kRbHalo / 2 && gcx < nc && gcy < nc) {
        const int64_t ci = (int64_t)gcy * nc + gcx;
        const T acc = (r[0][0] + r[0][1]) + (r[1][1] + r[1][0]);
        store_f(P.fc, ci, (P.cls_c[ci] & kClsUnknown) ? acc * (T)0.25 : (T)0, P.fc_bf16);
      }
    }
  }

  // ---------------------------------------------------------------- store the tile
#pragma unroll
  for (int j = 0; j < RW; ++j) {
    const int y = warp * RW + j, gy = y0 + y, p = j & 1;
    if (y < kRbHalo || y >= SY - kRbHalo || lane < kRbHalo / 2 || lane >= kRbKW - kRbHalo / 2) continue;
    if (gy >= n || gx >= n) continue;
    const int64_t g = (int64_t)gy * n + gx;
    const T a = p ? ub[j] : ur[j], b = p ? ur[j] : ub[j];
    if (UP && P.z != nullptr) {
      double2 st;
      st.x = (double)a;
      st.y = (double)b;
      *(double2*)(P.z + g) = st;
    } else {
      T2 st;
      st.x = a;
      st.y = b;
      *(T2*)(P.u_out + g) = st;
    }
  }
}

}  // namespace iim
