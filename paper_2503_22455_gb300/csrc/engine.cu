// Batched solve engine (host side): slot table, work lists, the captured tick
// graph and the tile-shape autotuner.  The kernels are the grouped forms in
// operator.cu, multigrid.cu and krylov.cu; the per-tick protocol is described in
// engine.cuh.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "engine.cuh"

namespace iim {

void eng_operator_params(Problem& P, StencilCoef* C, GhostParams* GP, CorrectParams* CP);
void eng_init_scalars(Problem& P, cudaStream_t s);
size_t mg_tail_start(const Problem& P);
template <typename T>
TailParams<T> make_tail_params(Problem& P, size_t l0, T* u_out, size_t smem_limit, size_t* smem);

// persistent grid: as many blocks of the kernel as fit on the device at once
int eng_grid(const void* kernel, int threads, size_t smem) {
  static std::mutex mu;
  static int sms = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms <= 0) sms = kNumSMs;
    }
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  return nb * sms;
}

constexpr size_t kEngTailSmem = 64 * 1024;   // dynamic shared memory of the grouped tail
constexpr int kEngSizeClasses = 6;           // 2D level size classes of the autotuner

static int size_class(int n) {
  if (n <= 32) return 0;
  if (n <= 64) return 1;
  if (n <= 128) return 2;
  if (n <= 256) return 3;
  if (n <= 512) return 4;
  return 5;
}

struct Engine {
  int cap = 0;
  iim_options opt;
  cudaStream_t stream = nullptr;
  SlotDev* d_slots = nullptr;
  int* d_lists = nullptr;               // the host's lists
  int* d_dyn = nullptr;                 // this tick's lists (plan kernel)
  int* d_ctl = nullptr;                 // [0] unfinished slots, [1] tick budget, [2 + slot] done flags
  int* h_ctl = nullptr;                 // pinned mirror
  cudaEvent_t ev_run = nullptr;
  bool run_pending = false;
  std::vector<Problem*> prob;           // nullptr: free slot
  std::vector<SlotDev> h_slots;
  std::vector<int> h_lists;
  std::vector<int> reported;            // done already reported by poll
  std::vector<int> list_items;          // items per list (host copy)
  bool dirty = true;
  // captured run graph
  unsigned char present[kListCount];
  bool captured = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t kernels_per_tick = 0;
  int64_t ticks = 0;
  int last_max = 0;
  int shape_of_class[kEngSizeClasses];
  std::vector<EngMgStep> mg_steps;
};

static EngArgs eng_args(const Engine& E) {
  EngArgs A;
  A.slots = E.d_slots;
  A.lists = E.d_dyn;
  A.stat = E.d_lists;
  A.cap = E.cap;
  return A;
}

static void default_shapes(Engine& E) {
  // the single-problem choice: 32 x 8 tiles below 512, 64 x 16 from 512 up
  for (int c = 0; c < kEngSizeClasses; ++c) E.shape_of_class[c] = c >= 5 ? 3 : 0;
}

static int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// the slot's device descriptor
static void fill_slot(Engine& E, int si, Problem& P) {
  SlotDev sd;
  std::memset(&sd, 0, sizeof(sd));
  sd.role = kRoleIdle;
  sd.j = 0;
  sd.dim = P.g.dim;
  sd.w = P.w;
  sd.iface = P.desc.bc == IIM_BC_INTERFACE;
  sd.neumann = P.desc.bc == IIM_BC_NEUMANN;
  sd.g = P.g;
  sd.phase = P.phase;
  sd.status = P.d_status + 1;           // the per-solve word (set-up failures stay in word 0)
  eng_operator_params(P, &sd.C, &sd.GP, &sd.CP);
  sd.sc = P.sc;
  sd.V = P.V;
  sd.Z = P.Z;
  sd.x = P.x;
  sd.tmp = P.tmp;
  sd.b = P.b;
  sd.Npad = P.Npad;
  sd.partial = P.partial;
  sd.counter = P.counter;
  sd.red_blocks = P.red_blocks;
  sd.xup_blocks = std::min(4 * kNumSMs, std::max(1, cdiv(P.g.N, 4 * 256)));
  sd.nlev = (int)P.lv.size();
  sd.nfine = (int)mg_tail_start(P);
  for (int l = 0; l < sd.nlev; ++l) {
    sd.lev[l] = levk<float>(P.lv[l]);
    sd.u2[l] = (float*)P.lv[l].u2;
  }
  sd.inv_bp = (float)(1.0 / P.desc.beta_plus);
  sd.inv_bm = (float)(1.0 / P.desc.beta_minus);
  size_t smem = 0;
  sd.tail = make_tail_params<float>(P, (size_t)sd.nfine, nullptr, kEngTailSmem, &smem);
  E.h_slots[si] = sd;
}

static void build_lists(Engine& E) {
  std::vector<std::vector<std::pair<int, int>>> L(kListCount);
  for (int si = 0; si < E.cap; ++si) {
    Problem* pp = E.prob[si];
    if (!pp) continue;
    Problem& P = *pp;
    const SlotDev& sd = E.h_slots[si];
    L[kListAll].push_back({si, 1});
    L[kListXup].push_back({si, sd.xup_blocks});
    L[kListRed].push_back({si, sd.red_blocks});
    L[kListStencil + (P.g.dim - 2) * 2 + (P.w - 2)].push_back({si, cdiv(P.g.N, 4 * kEngThreads)});
    if (P.K_cap > 0) L[kListGhost + (P.w - 2)].push_back({si, cdiv((int64_t)P.K_cap * 8, 64)});
    if (P.aff_cap > 0) L[kListCorrect].push_back({si, cdiv(P.aff_cap, 64)});
    L[kListTail].push_back({si, 1});
    for (int d = 0; d < sd.nfine; ++d) {
      const Level& lv = P.lv[d];
      if (P.g.dim == 2) {
        const int shape = E.shape_of_class[size_class(lv.g.n)];
        int gx, gy;
        eng_mg2d_tile_items(lv.g.n, shape, &gx, &gy);
        L[kListMg2d + d * kEngShapes + shape].push_back({si, gx * gy});
      } else {
        const int64_t ncol = (lv.g.N / lv.g.n) * ((lv.g.n + 1) / 2);
        L[kList3dN + d].push_back({si, cdiv(lv.g.N, 256)});
        L[kList3dCol + d].push_back({si, cdiv(ncol, 256)});
        L[kList3dCoarse + d].push_back({si, cdiv(P.lv[d + 1].g.N, 256)});
      }
    }
  }
  const size_t stride = 2 * (size_t)E.cap + 2;
  E.h_lists.assign(eng_list_ints(E.cap), 0);
  E.list_items.assign(kListCount, 0);
  for (int k = 0; k < kListCount; ++k) {
    int* p = E.h_lists.data() + k * stride;
    p[0] = (int)L[k].size();
    int acc = 0;
    for (size_t e = 0; e < L[k].size(); ++e) {
      p[1 + e] = acc;
      p[2 + E.cap + e] = L[k][e].first;
      acc += L[k][e].second;
    }
    p[1 + L[k].size()] = acc;
    E.list_items[k] = acc;
  }
}

// the V-cycle as a sequence of grouped launches: 2D fine levels, 3D fine levels, the
// tail, then back up.  The ping-pong buffer of each 2D step (0 = u, 1 = u2) follows
// the single-problem V-cycle, which alternates the two at every fused kernel.
static void build_mg_program(Engine& E, const unsigned char* present) {
  E.mg_steps.clear();
  int d2 = 0, d3 = 0;
  for (int d = 0; d < kEngMaxDepth; ++d) {
    for (int sh = 0; sh < kEngShapes; ++sh)
      if (present[kListMg2d + d * kEngShapes + sh]) d2 = d + 1;
    if (present[kList3dN + d]) d3 = d + 1;
  }
  const int nu1 = E.opt.nu1, nu2 = E.opt.nu2;
  // kernels of one fine level (the same at every depth) and their buffers: A starts as u
  struct Sel { int mode, in, out; };
  std::vector<Sel> down, up;
  int A = 0, B = 1;
  if (nu1 == 2 && nu2 == 2) {
    down.push_back({5, -1, A});                   // both pre-smoothing sweeps + restriction
    up.push_back({6, A, B});                      // correction + both post-smoothing sweeps
  } else {
    down.push_back({0, -1, A});
    for (int it = 1; it < nu1 - 1; ++it) { down.push_back({4, A, B}); std::swap(A, B); }
    down.push_back({1, A, B});
    std::swap(A, B);
    up.push_back({2, A, B});
    std::swap(A, B);
    for (int it = 1; it < nu2 - 1; ++it) { up.push_back({4, A, B}); std::swap(A, B); }
    up.push_back({3, A, B});
  }
  const int res = B;                              // the level's result
  auto add2 = [&](int d, const Sel& s) {
    for (int sh = 0; sh < kEngShapes; ++sh) {
      if (!present[kListMg2d + d * kEngShapes + sh]) continue;
      EngMgStep st{0, s.mode, d, sh, s.in < 0 ? 0 : s.in, s.out, res, 0};
      E.mg_steps.push_back(st);
    }
  };
  for (int d = 0; d < d2; ++d)
    for (const Sel& st : down) add2(d, st);
  auto add3 = [&](int kind3, int d, int colour) {
    EngMgStep st{2 + kind3, 0, d, 0, 0, 0, 0, colour};
    E.mg_steps.push_back(st);
  };
  if (d3 > 0) add3(0, 0, 0);
  for (int d = 0; d < d3; ++d) {
    add3(1, d, 0);
    for (int it = 0; it < nu1; ++it)
      for (int c = 0; c < 2; ++c) add3(2, d, c);
    add3(3, d, 0);
  }
  if (present[kListTail]) E.mg_steps.push_back(EngMgStep{1, 0, 0, 0, 0, 0, 0, 0});
  for (int d = d2 - 1; d >= 0; --d)
    for (const Sel& st : up) add2(d, st);
  for (int d = d3 - 1; d >= 0; --d) {
    add3(4, d, 0);
    for (int it = 0; it < nu2; ++it)
      for (int c = 0; c < 2; ++c) add3(2, d, c);
  }
  if (d3 > 0) add3(5, 0, 0);
}

static void enqueue_mg(Engine& E, cudaStream_t s) {
  const EngArgs A = eng_args(E);
  for (const EngMgStep& st : E.mg_steps) eng_launch_mg(A, st, kEngTailSmem, s);
}

static void enqueue_tick(Engine& E, cudaGraphConditionalHandle h, int use_cond, cudaStream_t s) {
  const EngArgs A = eng_args(E);
  eng_launch_krylov_head(A, E.d_dyn, s);
  enqueue_mg(E, s);
  eng_launch_apply(A, E.present, s);
  eng_launch_krylov_tail(A, E.d_ctl, h, use_cond, s);
}

static iim_status capture(Engine& E) {
  if (E.exec) cudaGraphExecDestroy(E.exec);
  if (E.graph) cudaGraphDestroy(E.graph);
  E.exec = nullptr;
  E.graph = nullptr;
  build_mg_program(E, E.present);
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return IIM_ERR_CUDA;
  cudaGraph_t g;
  cudaGraphCreate(&g, 0);
  cudaGraphConditionalHandle h;
  cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) != cudaSuccess) {
    cudaStreamDestroy(s);
    set_error("engine: conditional node");
    return IIM_ERR_CUDA;
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  const int64_t l0 = iim_launch_count();
  enqueue_tick(E, h, 1, s);
  E.kernels_per_tick = iim_launch_count() - l0;
  cudaStreamEndCapture(s, &body);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaGraphInstantiate(&E.exec, g, 0);
  cudaStreamDestroy(s);
  E.graph = g;
  if (e != cudaSuccess) {
    set_error(std::string("engine graph: ") + cudaGetErrorString(e));
    return IIM_ERR_CUDA;
  }
  E.captured = true;
  return IIM_OK;
}

// upload the lists; capture again when a list the graph does not launch became non-empty
static iim_status sync_lists(Engine& E) {
  if (!E.dirty) return IIM_OK;
  build_lists(E);
  bool need = !E.captured;
  for (int k = 0; k < kListCount; ++k) {
    const unsigned char p = E.list_items[k] > 0;
    if (p && !E.present[k]) need = true;
  }
  if (need)
    for (int k = 0; k < kListCount; ++k) E.present[k] = E.present[k] || E.list_items[k] > 0;
  cudaMemcpyAsync(E.d_lists, E.h_lists.data(), sizeof(int) * E.h_lists.size(), cudaMemcpyHostToDevice, E.stream);
  E.dirty = false;
  if (!need) return IIM_OK;
  if (!E.opt.use_graph) {
    build_mg_program(E, E.present);
    E.captured = true;
    return IIM_OK;
  }
  return capture(E);
}

static iim_status eng_cuda(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return IIM_ERR_CUDA;
  }
  return IIM_OK;
}

static void destroy_engine(Engine* E) {
  if (E->stream) cudaStreamSynchronize(E->stream);
  if (E->exec) cudaGraphExecDestroy(E->exec);
  if (E->graph) cudaGraphDestroy(E->graph);
  if (E->d_slots) cudaFree(E->d_slots);
  if (E->d_lists) cudaFree(E->d_lists);
  if (E->d_dyn) cudaFree(E->d_dyn);
  if (E->d_ctl) cudaFree(E->d_ctl);
  if (E->h_ctl) cudaFreeHost(E->h_ctl);
  if (E->ev_run) cudaEventDestroy(E->ev_run);
  delete E;
}

}  // namespace iim

using namespace iim;

struct iim_problem {
  Problem P;
};
struct iim_engine {
  Engine* E;
};

extern "C" {

iim_status iim_engine_create(const iim_options* opt, int max_slots, void* stream, iim_engine** out) {
  if (!opt || !out || max_slots < 1 || max_slots > (1 << 16)) return IIM_ERR_INVALID_ARG;
  *out = nullptr;
  if ((opt->mg_precision != IIM_MG_FP32 && opt->mg_precision != IIM_MG_FP32_BF16R) || opt->nu1 < 2 || opt->nu2 < 2) {
    set_error("the engine runs the FP32 multigrid with nu1, nu2 >= 2");
    return IIM_ERR_INVALID_ARG;
  }
  Engine* E = new Engine();
  E->cap = max_slots;
  E->opt = *opt;
  E->stream = (cudaStream_t)stream;
  E->prob.assign(max_slots, nullptr);
  E->h_slots.resize(max_slots);
  E->reported.assign(max_slots, 0);
  std::memset(E->present, 0, sizeof(E->present));
  default_shapes(*E);
  bool ok = cudaMalloc(&E->d_slots, sizeof(SlotDev) * (size_t)max_slots) == cudaSuccess &&
            cudaMalloc(&E->d_lists, sizeof(int) * eng_list_ints(max_slots)) == cudaSuccess &&
            cudaMalloc(&E->d_dyn, sizeof(int) * eng_dyn_ints(max_slots)) == cudaSuccess &&
            cudaMalloc(&E->d_ctl, sizeof(int) * (2 + (size_t)max_slots)) == cudaSuccess &&
            cudaMallocHost(&E->h_ctl, sizeof(int) * (2 + (size_t)max_slots)) == cudaSuccess &&
            cudaEventCreateWithFlags(&E->ev_run, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    set_error("engine: device allocation failed");
    destroy_engine(E);
    return IIM_ERR_BUDGET;
  }
  cudaMemsetAsync(E->d_lists, 0, sizeof(int) * eng_list_ints(max_slots), E->stream);
  cudaMemsetAsync(E->d_dyn, 0, sizeof(int) * eng_dyn_ints(max_slots), E->stream);
  cudaMemsetAsync(E->d_ctl, 0, sizeof(int) * (2 + (size_t)max_slots), E->stream);
  std::memset(E->h_ctl, 0, sizeof(int) * (2 + (size_t)max_slots));
  iim_status st = eng_cuda("engine create");
  if (st != IIM_OK) {
    destroy_engine(E);
    return st;
  }
  *out = new iim_engine{E};
  return IIM_OK;
}

void iim_engine_destroy(iim_engine* H) {
  if (!H) return;
  destroy_engine(H->E);
  delete H;
}

iim_status iim_engine_admit(iim_engine* H, iim_problem* p, const double* x0_dev, int* slot) {
  if (!H || !p) return IIM_ERR_INVALID_ARG;
  Engine& E = *H->E;
  Problem& P = p->P;
  if (P.opt.mg_precision == IIM_MG_FP64 || P.opt.nu1 != E.opt.nu1 || P.opt.nu2 != E.opt.nu2) {
    set_error("engine: the problem's multigrid options differ from the engine's");
    return IIM_ERR_INVALID_ARG;
  }
  if (P.aug) {
    set_error("engine: pure Neumann problems (augmented system) are solved by iim_solve only");
    return IIM_ERR_INVALID_ARG;
  }
  if (P.opt.cycle != IIM_CYCLE_V || P.opt.krylov != IIM_KRYLOV_FGMRES) {
    set_error("engine: W-cycles and left-preconditioned GMRES are solved by iim_solve only");
    return IIM_ERR_INVALID_ARG;
  }
  if ((int)mg_tail_start(P) > kEngMaxDepth) {
    set_error("engine: too many fine multigrid levels");
    return IIM_ERR_INVALID_ARG;
  }
  {
    size_t smem = 0;
    make_tail_params<float>(P, mg_tail_start(P), nullptr, kEngTailSmem, &smem);
    size_t base = 0;
    for (size_t l = mg_tail_start(P); l < P.lv.size(); ++l) base += (size_t)P.lv[l].g.N * 16;
    if (base > kEngTailSmem) {
      set_error("engine: coarse levels too large for the tail kernel");
      return IIM_ERR_INVALID_ARG;
    }
  }
  for (int si = 0; si < E.cap; ++si)
    if (E.prob[si] == &P) {
      set_error("engine: problem already admitted");
      return IIM_ERR_INVALID_ARG;
    }
  int si = -1;
  for (int k = 0; k < E.cap; ++k)
    if (!E.prob[k]) { si = k; break; }
  if (si < 0) {
    set_error("engine: no free slot");
    return IIM_ERR_CAPACITY;
  }
  // the problem's own stream (set-up, data) comes first
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, P.stream);
  cudaStreamWaitEvent(E.stream, ev, 0);
  cudaEventDestroy(ev);
  if (x0_dev) cudaMemcpyAsync(P.x, x0_dev, sizeof(double) * P.g.N, cudaMemcpyDeviceToDevice, E.stream);
  else cudaMemsetAsync(P.x, 0, sizeof(double) * P.g.N, E.stream);
  cudaMemsetAsync(P.d_status + 1, 0, sizeof(int), E.stream);
  eng_init_scalars(P, E.stream);
  fill_slot(E, si, P);
  cudaMemcpyAsync(E.d_slots + si, &E.h_slots[si], sizeof(SlotDev), cudaMemcpyHostToDevice, E.stream);
  cudaMemsetAsync(E.d_ctl + 2 + si, 0, sizeof(int), E.stream);
  E.h_ctl[2 + si] = 0;
  E.prob[si] = &P;
  E.reported[si] = 0;
  E.dirty = true;
  if (slot) *slot = si;
  return eng_cuda("engine admit");
}

// Run up to max_ticks ticks (one graph launch; the device stops early when every
// slot has finished).  Asynchronous: iim_engine_poll reports the outcome.
iim_status iim_engine_run(iim_engine* H, int max_ticks) {
  if (!H || max_ticks < 1) return IIM_ERR_INVALID_ARG;
  Engine& E = *H->E;
  bool any = false;
  for (int si = 0; si < E.cap; ++si) any = any || E.prob[si];
  if (!any) return IIM_OK;
  iim_status st = sync_lists(E);
  if (st != IIM_OK) return st;
  cudaMemcpyAsync(E.d_ctl + 1, &max_ticks, sizeof(int), cudaMemcpyHostToDevice, E.stream);
  if (E.opt.use_graph) {
    cudaGraphLaunch(E.exec, E.stream);
    note_launch();
  } else {
    // the same ticks as separate launches (for kernel-level profiling): the host reads
    // the unfinished-slot count after every tick
    for (int t = 0; t < max_ticks; ++t) {
      enqueue_tick(E, 0, 0, E.stream);
      cudaMemcpyAsync(E.h_ctl, E.d_ctl, sizeof(int) * 2, cudaMemcpyDeviceToHost, E.stream);
      cudaStreamSynchronize(E.stream);
      if (E.h_ctl[0] == 0) break;
    }
    E.kernels_per_tick = 0;
  }
  cudaMemcpyAsync(E.h_ctl, E.d_ctl, sizeof(int) * (2 + (size_t)E.cap), cudaMemcpyDeviceToHost, E.stream);
  cudaEventRecord(E.ev_run, E.stream);
  E.run_pending = true;
  E.last_max = max_ticks;
  return eng_cuda("engine run");
}

// Outcome of the last run: *live = unfinished slots, done[0 .. *ndone) = slots that
// finished since the previous poll.  wait = 0 returns IIM_ERR_TIMEOUT while the run is
// still on the device (nothing is reported then).
iim_status iim_engine_poll(iim_engine* H, int wait, int* live, int* done, int* ndone, int64_t* ticks_run) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Engine& E = *H->E;
  if (ndone) *ndone = 0;
  if (E.run_pending) {
    if (wait) cudaEventSynchronize(E.ev_run);
    else if (cudaEventQuery(E.ev_run) == cudaErrorNotReady) return IIM_ERR_TIMEOUT;
    iim_status st = eng_cuda("engine poll");
    if (st != IIM_OK) return st;
    E.run_pending = false;
    E.ticks += E.last_max - E.h_ctl[1];
  }
  if (live) *live = E.h_ctl[0];
  int nd = 0;
  for (int si = 0; si < E.cap; ++si) {
    if (!E.prob[si] || E.reported[si] || !E.h_ctl[2 + si]) continue;
    E.reported[si] = 1;
    if (done) done[nd] = si;
    ++nd;
  }
  if (ndone) *ndone = nd;
  if (ticks_run) *ticks_run = E.ticks;
  return IIM_OK;
}

// Take a slot out of the engine: its solution to x_dev (may be NULL) and its
// solve summary.  The problem itself stays with the caller.  Synchronises the
// engine's stream.
iim_status iim_engine_release(iim_engine* H, int slot, double* x_dev, iim_solve_info* info) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Engine& E = *H->E;
  if (slot < 0 || slot >= E.cap || !E.prob[slot]) return IIM_ERR_INVALID_ARG;
  Problem& P = *E.prob[slot];
  if (x_dev) cudaMemcpyAsync(x_dev, P.x, sizeof(double) * P.g.N, cudaMemcpyDeviceToDevice, E.stream);
  SolverScalars h;
  cudaMemcpyAsync(&h, P.sc, sizeof(SolverScalars), cudaMemcpyDeviceToHost, E.stream);
  int stw[2] = {0, 0};
  cudaMemcpyAsync(stw, P.d_status, sizeof(stw), cudaMemcpyDeviceToHost, E.stream);
  cudaStreamSynchronize(E.stream);
  iim_status st = eng_cuda("engine release");
  if (st != IIM_OK) return st;
  iim_solve_info tmp;
  std::memset(&tmp, 0, sizeof(tmp));
  tmp.iters = h.iters;
  tmp.restarts = h.restarts;
  tmp.converged = h.converged;
  tmp.relres = h.relres;
  tmp.kernels = 0;
  iim_status dst = (iim_status)(stw[0] ? stw[0] : stw[1]);
  if (dst == IIM_OK && !h.converged) dst = h.done ? IIM_ERR_NOT_CONVERGED : IIM_ERR_TIMEOUT;
  tmp.status = dst;
  if (info) *info = tmp;
  // a later occupant of the slot must not see this one's done flag
  cudaMemsetAsync(E.d_ctl + 2 + slot, 0, sizeof(int), E.stream);
  E.h_ctl[2 + slot] = 0;
  E.prob[slot] = nullptr;
  E.reported[slot] = 0;
  E.dirty = true;
  return eng_cuda("engine release");
}

// Grouped launches in one tick graph, and ticks run so far.
iim_status iim_engine_stats(iim_engine* H, int64_t* kernels_per_tick, int64_t* ticks) {
  if (!H) return IIM_ERR_INVALID_ARG;
  if (kernels_per_tick) *kernels_per_tick = H->E->kernels_per_tick;
  if (ticks) *ticks = H->E->ticks;
  return IIM_OK;
}

// Tile shape of the fused 2D smoothing kernels per level size class (n <= 32, 64, 128,
// 256, 512, larger): 0 = 32x8, 1 = 64x8, 2 = 32x16, 3 = 64x16.  NULL restores the default.
iim_status iim_engine_set_shapes(iim_engine* H, const int* shape_of_class) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Engine& E = *H->E;
  if (!shape_of_class) default_shapes(E);
  else
    for (int c = 0; c < kEngSizeClasses; ++c) {
      if (shape_of_class[c] < 0 || shape_of_class[c] >= kEngShapes) return IIM_ERR_INVALID_ARG;
      E.shape_of_class[c] = shape_of_class[c];
    }
  E.dirty = true;
  return IIM_OK;
}

iim_status iim_engine_get_shapes(iim_engine* H, int* shape_of_class) {
  if (!H || !shape_of_class) return IIM_ERR_INVALID_ARG;
  for (int c = 0; c < kEngSizeClasses; ++c) shape_of_class[c] = H->E->shape_of_class[c];
  return IIM_OK;
}

// Autotuner: for every 2D level size class in use, time the whole grouped V-cycle of
// the admitted slots with each tile shape and keep the fastest.  Runs V-cycles on
// Krylov vector 0 of every slot, so it must come before the first tick after the
// slots were admitted (it is refused once any admitted slot has started).
iim_status iim_engine_autotune(iim_engine* H, int reps, double* best_ms) {
  if (!H || reps < 1) return IIM_ERR_INVALID_ARG;
  Engine& E = *H->E;
  if (E.run_pending) cudaEventSynchronize(E.ev_run);
  E.run_pending = false;
  // only fresh slots: the scalars' first flag is still set
  for (int si = 0; si < E.cap; ++si) {
    if (!E.prob[si]) continue;
    SolverScalars h;
    cudaMemcpyAsync(&h, E.prob[si]->sc, sizeof(SolverScalars), cudaMemcpyDeviceToHost, E.stream);
    cudaStreamSynchronize(E.stream);
    if (!h.first) {
      set_error("engine autotune: a slot has already started");
      return IIM_ERR_INVALID_ARG;
    }
  }
  bool used[kEngSizeClasses] = {false};
  for (int si = 0; si < E.cap; ++si) {
    Problem* P = E.prob[si];
    if (!P || P->g.dim != 2) continue;
    const int nf = (int)mg_tail_start(*P);
    for (int d = 0; d < nf; ++d) used[size_class(P->lv[d].g.n)] = true;
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const EngArgs A = eng_args(E);
  auto time_program = [&]() -> float {
    E.dirty = true;
    build_lists(E);
    unsigned char pres[kListCount];
    for (int k = 0; k < kListCount; ++k) pres[k] = E.list_items[k] > 0;
    build_mg_program(E, pres);
    cudaMemcpyAsync(E.d_lists, E.h_lists.data(), sizeof(int) * E.h_lists.size(), cudaMemcpyHostToDevice, E.stream);
    eng_launch_plan(A, E.d_dyn, 1, E.stream);          // every slot ITER at j = 0
    enqueue_mg(E, E.stream);
    cudaEventRecord(a, E.stream);
    for (int r = 0; r < reps; ++r) enqueue_mg(E, E.stream);
    cudaEventRecord(b, E.stream);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    return ms / reps;
  };
  float best_all = time_program();
  for (int c = 0; c < kEngSizeClasses; ++c) {
    if (!used[c]) continue;
    int best = E.shape_of_class[c];
    float bt = 1e30f;
    for (int sh = 0; sh < kEngShapes; ++sh) {
      E.shape_of_class[c] = sh;
      const float t = time_program();
      if (t < bt) { bt = t; best = sh; }
    }
    E.shape_of_class[c] = best;
    best_all = bt;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  // the next run rebuilds the lists (and the graph if the launches changed)
  E.dirty = true;
  E.captured = false;
  std::memset(E.present, 0, sizeof(E.present));
  if (best_ms) *best_ms = best_all;
  return eng_cuda("engine autotune");
}

}  // extern "C"
