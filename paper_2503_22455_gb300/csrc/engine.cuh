// Batched solve engine: many independent problems advanced together, one FGMRES
// step per "tick" (Sec. 4.1 iteration, Sec. 3.3 V-cycle, Sec. 2.3 operator).
//
// Every problem ("slot") keeps its whole state on the device: grids, multigrid
// hierarchy, Krylov basis and the FGMRES scalars.  A tick is a fixed sequence of
// persistent kernels.  Each kernel walks a work list of (slot, item) pairs, where an
// item is one thread block's share of that slot's work: the same block the
// single-problem kernel would run, so every slot computes bit for bit what a
// solve of that problem alone computes.  A plan kernel at the start of the tick
// gives every slot its role from its FGMRES state:
//   ITER     iteration j: z_j = M v_j, w = L z_j, orthogonalise, Givens step
//   RESTART  x += Z y, t = L x, v_0 = b - t, true-residual test (also the start)
//   IDLE     finished
// and the kernels skip items of slots whose role does not use them.  The lists
// live at fixed device addresses, so the captured tick graph stays valid while
// slots join and leave; the host only rewrites the lists.
#pragma once

#include "kernels.cuh"
#include "mg_fused.cuh"

namespace iim {

constexpr int kRoleIdle = 0, kRoleIter = 1, kRoleRestart = 2;
constexpr int kEngMaxDepth = 8;               // fine (tile-kernel) levels per slot
constexpr int kEngShapes = 4;                 // 2D smoothing tile shapes the autotuner picks from
constexpr int kEngThreads = 256;

// 2D tile shapes (TX x TY) of the fused smoothing kernels
constexpr int kShapeTX[kEngShapes] = {32, 64, 32, 64};
constexpr int kShapeTY[kEngShapes] = {8, 8, 16, 16};

// work lists
enum EngList {
  kListAll = 0,                                // every slot, one item
  kListXup,                                    // x += Z y
  kListRed,                                    // reductions: red_blocks items
  kListStencil,                                // + (dim - 2) * 2 + (w - 2): four lists
  kListGhost = kListStencil + 4,               // + (w - 2): two lists
  kListCorrect = kListGhost + 2,
  kListTail,                                   // one item
  kListMg2d,                                   // + depth * kEngShapes + shape
  kList3dN = kListMg2d + kEngMaxDepth * kEngShapes,   // + depth: ceil(N_d / 256)
  kList3dCol = kList3dN + kEngMaxDepth,        // + depth: one colour of level d
  kList3dCoarse = kList3dCol + kEngMaxDepth,   // + depth: ceil(N_{d+1} / 256)
  kListCount = kList3dCoarse + kEngMaxDepth
};

// Per-tick lists: the plan kernel copies every static list above, keeping only the
// slots whose role this tick uses it, plus three lists that select by role alone.
enum EngDynList { kDynAllIter = kListCount, kDynAllRestart, kDynRedRestart, kDynCount };
constexpr int kMaskIter = 1 << kRoleIter, kMaskRestart = 1 << kRoleRestart;

// roles that use dynamic list k
__host__ __device__ inline int eng_list_mask(int k) {
  if (k == kListXup || k == kDynAllRestart || k == kDynRedRestart) return kMaskRestart;
  if (k == kListAll || (k >= kListStencil && k <= kListCorrect)) return kMaskIter | kMaskRestart;
  return kMaskIter;                            // reductions of the iteration, Arnoldi, the V-cycle
}
// the static list a dynamic list is drawn from
__host__ __device__ inline int eng_list_source(int k) {
  if (k == kDynAllIter || k == kDynAllRestart) return kListAll;
  if (k == kDynRedRestart) return kListRed;
  return k;
}

// Everything a tick needs about one problem.  Written by the host at admission,
// except role and j, which the plan kernel sets at the start of every tick.
struct SlotDev {
  int role, j;
  int dim, w, iface, neumann;
  GridView g;
  const uint8_t* phase;
  int* status;
  StencilCoef C;
  GhostParams GP;                              // homogeneous (with_data = 0); G is the slot's
  CorrectParams CP;
  SolverScalars* sc;
  double *V, *Z, *x, *tmp, *b;
  int64_t Npad;
  double* partial;
  unsigned int* counter;
  int red_blocks, xup_blocks;
  int nlev, nfine;                             // levels nfine .. nlev-1 run in the tail
  LevelK<float> lev[kMaxLevels];
  float* u2[kMaxLevels];
  float inv_bp, inv_bm;
  TailParams<float> tail;                      // v, vscale and z are passed per tick
};

// list layout (ints): [0] count, [1 .. count+1] item prefix, [2 + cap ..] slot of each entry.
// `lists` are this tick's lists (written by the plan kernel), `stat` the host's.
struct EngArgs {
  SlotDev* slots;
  const int* lists;
  const int* stat;
  int cap;
  __device__ const int* list(int k) const { return lists + (size_t)k * (2 * cap + 2); }
  __device__ const int* slist(int k) const { return stat + (size_t)k * (2 * cap + 2); }
};

inline size_t eng_list_ints(int cap) { return (size_t)kListCount * (2 * cap + 2); }
inline size_t eng_dyn_ints(int cap) { return (size_t)kDynCount * (2 * cap + 2); }

// Persistent loop over the items of list k: f(slot, item-within-slot).  Block b
// takes the contiguous items [b*per, (b+1)*per) (items are ordered by slot), finds
// the entry of its first item with one parallel search through shared memory, then
// walks forward.  Every thread of the block takes part; the block synchronises
// between items, so shared memory can be reused by the next item.
template <class F>
__device__ __forceinline__ void eng_for_items(const EngArgs& A, int k, F&& f) {
  const int* L = A.list(k);
  const int count = L[0];
  if (count <= 0) return;
  const int* pre = L + 1;
  const int* slot = L + 2 + A.cap;
  const int total = pre[count];
  const int per = (total + gridDim.x - 1) / gridDim.x;
  int item = blockIdx.x * per;
  const int end = min(total, item + per);
  if (item >= end) return;
  __shared__ int s_entry;
  {
    // the entry e with pre[e] <= item < pre[e + 1]: first the chunk of entries, then the entry
    const int nt = blockDim.x;
    const int step = (count + nt - 1) / nt;
    int lo = 0;
    if (step > 1) {
      if (threadIdx.x == 0) s_entry = 0;
      __syncthreads();
      const int c0 = threadIdx.x * step;
      if (c0 < count && pre[c0] <= item && (c0 + step >= count || pre[c0 + step] > item)) s_entry = c0;
      __syncthreads();
      lo = s_entry;
      __syncthreads();
    }
    const int span = step > 1 ? step : count;          // entries of the chunk (all of them if one chunk)
    for (int t = threadIdx.x; t < span; t += nt) {
      const int e = lo + t;
      if (e < count && pre[e] <= item && pre[e + 1] > item) s_entry = e;
    }
    __syncthreads();
  }
  int e = s_entry;
  int first = pre[e], next = pre[e + 1];
  for (; item < end; ++item) {
    while (item >= next) {
      ++e;
      first = next;
      next = pre[e + 1];
    }
    f(slot[e], item - first);
    __syncthreads();
  }
}

// pointers of the operator apply for the slot's role this tick
__device__ __forceinline__ void eng_apply_io(const SlotDev& s, const double*& u, double*& w) {
  if (s.role == kRoleIter) {
    u = s.Z + (size_t)s.j * s.Npad;
    w = s.V + (size_t)(s.j + 1) * s.Npad;
  } else {
    u = s.x;
    w = s.tmp;
  }
}

// host-side launchers (one per translation unit that owns the kernel bodies)
int eng_grid(const void* kernel, int threads, size_t smem);
void eng_launch_apply(const EngArgs& A, const unsigned char* present, cudaStream_t s);
void eng_launch_plan(const EngArgs& A, int* dyn, int force_iter, cudaStream_t s);
void eng_launch_krylov_head(const EngArgs& A, int* dyn, cudaStream_t s);
void eng_launch_krylov_tail(const EngArgs& A, int* ctl, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s);
struct EngMgStep {
  int kind;          // 0: 2D tile kernel (mode), 1: tail, 2..: 3D kernels
  int mode, depth, shape;
  int in_sel, out_sel, res_sel, colour;
};
void eng_launch_mg(const EngArgs& A, const EngMgStep& st, size_t tail_smem, cudaStream_t s);
void eng_mg2d_tile_items(int n, int shape, int* gx, int* gy);

}  // namespace iim
