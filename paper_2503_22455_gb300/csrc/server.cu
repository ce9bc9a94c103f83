// Request loop over the batched engine: requests are admitted while the device
// memory they need fits a budget, created and set up by a pool of host threads on
// their own streams while the engine runs the resident solves, join the engine at
// the next run (continuous batching at the granularity of a run of a few ticks) and
// leave it when their solve ends.  Latency is measured from submission to the
// moment the solution is on the host.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "kernels.cuh"

namespace iim {

// Device bytes a problem of this descriptor will hold, before it exists: the
// per-node workspace of create exactly, and the fits for a body whose control-point
// count is about 3n (2D) or 1.5 n^2 (3D).  It only decides when to try an
// admission; the exact size, known once the problem exists, is what is charged.
static size_t estimate_bytes(const iim_problem_desc& d, const iim_options& o) {
  const double N = (double)d.n * d.n * (d.dim == 3 ? d.n : 1);
  const double vec = 8.0 * (o.restart + 1 + (o.krylov == IIM_KRYLOV_GMRES_LEFT ? 1 : o.restart) + 2);   // V, Z, x, tmp
  const double grid = 1.0 + 8.0 * d.dim + 8.0 + 8.0;          // phase, edge flags/ids, affected flags/ids, b
  const double mg = (d.dim == 2 ? 4.0 / 3.0 : 8.0 / 7.0) * (1.0 + 12.0 + 12.0);   // phase, aux/flag/idx, u/u2/f
  const double K = d.dim == 2 ? 3.0 * d.n : 1.5 * (double)d.n * d.n;
  const int w = d.order / 2, rc = rows_cap(d.dim, d.order);
  const double nfit = 1.25 * K * (d.bc == IIM_BC_INTERFACE ? 2 : 1) + 64;
  const double fit = nfit * (4.0 * rc + 8.0 * (w + 1) * rc + 16.0 * w + 64.0) + K * 160.0;
  return (size_t)(N * (vec + grid + mg) + fit) + (1 << 20);
}

using Clock = std::chrono::steady_clock;

}  // namespace iim
struct iim_problem {
  iim::Problem P;
};
namespace iim {

enum ReqState { kQueued = 0, kCreating, kNeedData, kReady, kRunning, kRetired, kFinished, kFailed };

struct Request {
  int64_t id = 0;
  iim_problem_desc desc;
  std::vector<double> geom_coef;  // the request's own copy of a Fourier curve's coefficients
  bool reuse = false;             // takes a retired problem of the same kind from the pool
  bool cancel = false;            // cancelled while being created or running: ends without a solution
  size_t freed_bytes = 0;         // a pooled problem the worker had to destroy (reuse failed)
  double t_submit = 0, t_done = 0;
  int state = kQueued;
  iim_problem* prob = nullptr;
  cudaStream_t stream = nullptr;
  size_t bytes = 0;
  size_t reserved = 0;           // budget held while it is being created
  size_t known_bytes = 0;        // exact size once the request has been created
  iim_status create_status = IIM_OK;
  int slot = -1;
  iim_solve_info info;
  std::vector<double> x;
  iim_status error = IIM_OK;
};

// Retired problems kept for reuse: a request of the same kind (dimension, size, conditions,
// order, geometry kind, side, coefficients) takes one and re-runs its set-up in place with
// its own geometry parameters, keeping the allocation, the stream and the solve graph.
struct PoolKey {
  int dim, n, bc, box_bc, order, kind, plus_inside;
  double bp, bm;
  bool operator==(const PoolKey& o) const {
    return dim == o.dim && n == o.n && bc == o.bc && box_bc == o.box_bc && order == o.order && kind == o.kind &&
           plus_inside == o.plus_inside && bp == o.bp && bm == o.bm;
  }
};
struct PoolEntry {
  PoolKey key;
  iim_problem* prob;
  cudaStream_t stream;
  size_t bytes;
  int64_t stamp;
};

static bool poolable(const iim_problem_desc& d) {
  // analytic bodies: their whole geometry is in geom_params (the set-up can change it in place)
  return d.geom_kind != IIM_GEOM_FOURIER && d.geom_kind != IIM_GEOM_LEVELSET_GRID;
}
static PoolKey pool_key(const iim_problem_desc& d) {
  return PoolKey{d.dim, d.n, d.bc, d.box_bc, d.order, d.geom_kind, d.plus_inside, d.beta_plus, d.beta_minus};
}

struct Server {
  iim_options opt;
  std::vector<PoolEntry> pool;   // retired problems (their bytes stay counted in in_use)
  int64_t pool_stamp = 0, pool_hits = 0, pool_misses = 0, pool_evicted = 0;
  bool pooling = false;          // reuse of retired problems: off unless the caller asks
  size_t budget = 0, in_use = 0, peak = 0;
  int max_slots = 0, ticks_per_run = 1;
  iim_engine* engine = nullptr;
  cudaStream_t stream = nullptr;
  std::vector<cudaStream_t> free_streams;
  std::map<int64_t, Request*> reqs;
  std::deque<Request*> queue;
  std::vector<Request*> slot_req;
  std::vector<int> done_buf;
  int64_t next_id = 1;
  bool run_in_flight = false;
  int resident = 0;
  int64_t runs = 0;
  int mode = 0;                  // 0: batched engine, 1: each request's solve graph on its own stream
  std::vector<Request*> running;  // mode 1
  // ids to report to the caller (kept until a step has room for them)
  std::deque<int64_t> note_need, note_fin;
  double t_step = 0, t_copy = 0, t_create = 0;   // host seconds: step calls, result copies, creation (workers)
  Clock::time_point t0;
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
  // creation workers
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> to_create;
  std::vector<Request*> created;
  bool stop = false;
  int device = 0;
  int creating = 0;
};

// worker: create the problem (allocation, set-up on the request's own stream, and the
// host waits inside create) away from the loop's thread
static void create_worker(Server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !S->to_create.empty(); });
      if (S->stop && S->to_create.empty()) return;
      r = S->to_create.front();
      S->to_create.pop_front();
    }
    const auto t = Clock::now();
    bool fresh = true;
    if (r->reuse && r->prob) {
      // re-run the set-up in place with this request's geometry, on the problem's own stream
      iim_status st = setup_direct(r->prob->P, r->desc.geom_params);
      if (st == IIM_OK) st = iim_status_get(r->prob);
      if (st == IIM_OK) {
        r->create_status = IIM_OK;
        fresh = false;
      } else {
        // capacity or geometry: give the problem up and create one for this request
        r->freed_bytes = r->prob->P.bytes;
        cudaStream_t keep = r->stream;
        iim_problem_destroy(r->prob);
        r->prob = nullptr;
        r->stream = keep;
        r->reuse = false;
      }
    }
    if (fresh) {
      r->create_status = iim_problem_create(&r->desc, &S->opt, r->stream, &r->prob);
      if (r->create_status != IIM_OK) r->prob = nullptr;
    }
    // streams mode: capture the request's solve graph here, off the loop's thread
    if (r->prob && fresh && S->mode == 1 && S->opt.use_graph) {
      r->create_status = krylov_build_graph(r->prob->P, r->prob->P.x);
      if (r->create_status != IIM_OK) {
        iim_problem_destroy(r->prob);
        r->prob = nullptr;
      }
    }
    const double dt = std::chrono::duration<double>(Clock::now() - t).count();
    std::lock_guard<std::mutex> lk(S->mu);
    S->t_create += dt;
    S->created.push_back(r);
  }
}

}  // namespace iim

using namespace iim;

struct iim_server {
  Server S;
};

static void free_problem(Server& S, Request* r, bool keep = false) {
  if (r->prob && keep && S.pooling && poolable(r->desc) && r->stream) {
    // the problem (and its stream, which its solve graph and set-up use) waits for a request
    // of the same kind; its bytes stay counted until it is reused or evicted
    S.pool.push_back(PoolEntry{pool_key(r->desc), r->prob, r->stream, r->bytes, ++S.pool_stamp});
    r->prob = nullptr;
    r->stream = nullptr;
    return;
  }
  if (r->prob) {
    iim_problem_destroy(r->prob);
    r->prob = nullptr;
    S.in_use -= r->bytes;
  }
  if (r->stream) S.free_streams.push_back(r->stream);
  r->stream = nullptr;
}

// free pooled problems, oldest first, until need more bytes fit the budget (or none is left)
static void pool_evict(Server& S, size_t need) {
  while (!S.pool.empty() && S.in_use + need > S.budget) {
    size_t old = 0;
    for (size_t k = 1; k < S.pool.size(); ++k)
      if (S.pool[k].stamp < S.pool[old].stamp) old = k;
    PoolEntry e = S.pool[old];
    S.pool[old] = S.pool.back();
    S.pool.pop_back();
    iim_problem_destroy(e.prob);
    S.in_use -= e.bytes;
    S.free_streams.push_back(e.stream);
    ++S.pool_evicted;
  }
}

// a request that holds no running work ends now, without a solution (IIM_ERR_TIMEOUT)
static void cancel_now(Server& S, Request* r) {
  if (r->state == kQueued) {
    for (auto it = S.queue.begin(); it != S.queue.end(); ++it)
      if (*it == r) { S.queue.erase(it); break; }
  }
  if (r->state == kNeedData) {
    for (auto it = S.note_need.begin(); it != S.note_need.end(); ++it)
      if (*it == r->id) { S.note_need.erase(it); break; }
  }
  free_problem(S, r);
  r->state = kFailed;
  r->error = IIM_ERR_TIMEOUT;
  r->info.status = IIM_ERR_TIMEOUT;
  r->t_done = S.now();
  S.note_fin.push_back(r->id);
}

// batched engine, no run in flight: release the cancelled slots (their solves stop here)
static void release_cancelled(Server& S, std::vector<Request*>& retired) {
  for (Request*& sr : S.slot_req) {
    Request* r = sr;
    if (!r || !r->cancel) continue;
    iim_engine_release(S.engine, r->slot, nullptr, &r->info);
    sr = nullptr;
    r->slot = -1;
    r->state = kRetired;
    --S.resident;
    retired.push_back(r);
  }
}

extern "C" {

iim_status iim_server_create(const iim_options* opt, size_t hbm_budget, int max_slots, int ticks_per_run,
                             int create_threads, iim_server** out) {
  if (!opt || !out || max_slots < 1 || ticks_per_run < 1 || hbm_budget == 0 || create_threads < 1 ||
      create_threads > 64)
    return IIM_ERR_INVALID_ARG;
  *out = nullptr;
  iim_server* H = new iim_server();
  Server& S = H->S;
  S.opt = *opt;
  S.budget = hbm_budget;
  S.max_slots = max_slots;
  S.ticks_per_run = ticks_per_run;
  S.t0 = Clock::now();
  if (cudaStreamCreateWithFlags(&S.stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete H;
    return IIM_ERR_CUDA;
  }
  iim_status st = iim_engine_create(opt, max_slots, S.stream, &S.engine);
  if (st != IIM_OK) {
    cudaStreamDestroy(S.stream);
    delete H;
    return st;
  }
  S.slot_req.assign(max_slots, nullptr);
  S.done_buf.assign(max_slots, 0);
  cudaGetDevice(&S.device);
  for (int k = 0; k < create_threads; ++k) S.workers.emplace_back(create_worker, &S);
  *out = H;
  return IIM_OK;
}

void iim_server_destroy(iim_server* H) {
  if (!H) return;
  Server& S = H->S;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stop = true;
    S.to_create.clear();
  }
  S.cv.notify_all();
  for (auto& t : S.workers) t.join();
  if (S.stream) cudaStreamSynchronize(S.stream);
  for (auto& kv : S.reqs) {
    Request* r = kv.second;
    if (r->slot >= 0) iim_engine_release(S.engine, r->slot, nullptr, nullptr);
    free_problem(S, r);
    delete r;
  }
  for (PoolEntry& e : S.pool) {
    iim_problem_destroy(e.prob);
    S.free_streams.push_back(e.stream);
  }
  S.pool.clear();
  iim_engine_destroy(S.engine);
  for (cudaStream_t s : S.free_streams) cudaStreamDestroy(s);
  cudaStreamDestroy(S.stream);
  delete H;
}

iim_status iim_server_set_pooling(iim_server* H, int on) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Server& S = H->S;
  S.pooling = on != 0;
  if (!S.pooling) pool_evict(S, S.budget + 1);       // frees every pooled problem
  return IIM_OK;
}

iim_status iim_server_pool_stats(iim_server* H, int64_t* hits, int64_t* misses, int64_t* evicted, int* pooled) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Server& S = H->S;
  if (hits) *hits = S.pool_hits;
  if (misses) *misses = S.pool_misses;
  if (evicted) *evicted = S.pool_evicted;
  if (pooled) *pooled = (int)S.pool.size();
  return IIM_OK;
}

iim_status iim_server_submit(iim_server* H, const iim_problem_desc* desc, int64_t* id) {
  if (!H || !desc || !id) return IIM_ERR_INVALID_ARG;
  Server& S = H->S;
  if (estimate_bytes(*desc, S.opt) > S.budget) {
    set_error("server: the request alone exceeds the memory budget");
    return IIM_ERR_BUDGET;
  }
  if (desc->geom_kind == IIM_GEOM_LEVELSET_GRID) {
    set_error("server: requests take analytic bodies or Fourier curves, not level sets on a grid");
    return IIM_ERR_INVALID_ARG;
  }
  if (desc->geom_kind == IIM_GEOM_FOURIER &&
      (!desc->geom_coef || desc->n_geom_coef < 3 || desc->n_geom_coef > 2 * IIM_MAX_FOURIER_MODES + 1)) {
    set_error("server: a Fourier curve needs 2 K + 1 coefficients, 1 <= K <= 16");
    return IIM_ERR_INVALID_ARG;
  }
  Request* r = new Request();
  r->id = S.next_id++;
  r->desc = *desc;
  if (desc->geom_kind == IIM_GEOM_FOURIER) {
    r->geom_coef.assign(desc->geom_coef, desc->geom_coef + desc->n_geom_coef);
    r->desc.geom_coef = r->geom_coef.data();
  } else {
    r->desc.geom_coef = nullptr;
    r->desc.n_geom_coef = 0;
  }
  r->desc.phi_dev = nullptr;
  r->t_submit = S.now();
  std::memset(&r->info, 0, sizeof(r->info));
  S.reqs[r->id] = r;
  S.queue.push_back(r);
  *id = r->id;
  return IIM_OK;
}

iim_status iim_server_step(iim_server* H, int64_t* need_data, int cap_need, int* n_need, int64_t* finished,
                           int cap_fin, int* n_fin) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Server& S = H->S;
  const auto t_enter = Clock::now();
  int nn = 0, nf = 0;
  std::vector<Request*> retired;
  // 1. finished solves: in streams mode, every running request whose solve graph is done
  if (S.mode == 1) {
    for (size_t k = 0; k < S.running.size();) {
      Request* r = S.running[k];
      if (cudaEventQuery(r->prob->P.ev1) == cudaErrorNotReady) { ++k; continue; }
      cudaGetLastError();
      solve_finish(r->prob->P, &r->info);
      r->state = kRetired;
      --S.resident;
      retired.push_back(r);
      S.running[k] = S.running.back();
      S.running.pop_back();
    }
  }
  // 1. the last run: release the slots that finished
  if (S.mode == 0 && S.run_in_flight) {
    int nd = 0;
    iim_status st = iim_engine_poll(S.engine, 0, nullptr, S.done_buf.data(), &nd, nullptr);
    if (st == IIM_OK) {
      S.run_in_flight = false;
      for (int k = 0; k < nd; ++k) {
        Request* r = S.slot_req[S.done_buf[k]];
        if (!r) continue;
        iim_engine_release(S.engine, r->slot, nullptr, &r->info);
        S.slot_req[r->slot] = nullptr;
        r->slot = -1;
        r->state = kRetired;
        --S.resident;
        retired.push_back(r);
      }
      release_cancelled(S, retired);
    } else if (st != IIM_ERR_TIMEOUT) {
      return st;
    }
  }
  if (S.mode == 0 && !S.run_in_flight) release_cancelled(S, retired);
  // 2 (streams mode). launch the solves of ready requests while slots are free
  if (S.mode == 1) {
    for (auto& kv : S.reqs) {
      Request* r = kv.second;
      if (r->state != kReady || S.resident >= S.max_slots) continue;
      iim_status st = solve_async(r->prob->P);
      if (st != IIM_OK) {
        r->state = kFailed;
        r->error = st;
        r->t_done = S.now();
        free_problem(S, r);
        S.note_fin.push_back(r->id);
        continue;
      }
      r->state = kRunning;
      ++S.resident;
      S.running.push_back(r);
    }
  }
  // 2. join the requests whose data are set, and launch the next run
  if (S.mode == 0 && !S.run_in_flight) {
    for (auto& kv : S.reqs) {
      Request* r = kv.second;
      if (r->state != kReady) continue;
      int slot = -1;
      iim_status st = iim_engine_admit(S.engine, r->prob, nullptr, &slot);
      if (st == IIM_ERR_CAPACITY) break;
      if (st != IIM_OK) {
        r->state = kFailed;
        r->error = st;
        r->t_done = S.now();
        free_problem(S, r);
        S.note_fin.push_back(r->id);
        continue;
      }
      r->slot = slot;
      r->state = kRunning;
      S.slot_req[slot] = r;
      ++S.resident;
    }
    if (S.resident > 0) {
      iim_status st = iim_engine_run(S.engine, S.ticks_per_run);
      if (st != IIM_OK) return st;
      S.run_in_flight = true;
      ++S.runs;
    }
  }
  // 3. solutions of the retired requests to the host (beside the new run), then free
  for (Request* r : retired) {
    if (r->cancel) {
      r->info.status = IIM_ERR_TIMEOUT;
      r->info.converged = 0;
      r->t_done = S.now();
      r->state = kFailed;
      r->error = IIM_ERR_TIMEOUT;
      free_problem(S, r);
      S.note_fin.push_back(r->id);
      continue;
    }
    Problem& P = r->prob->P;
    const auto tc = Clock::now();
    r->x.resize((size_t)P.g.N);
    cudaMemcpyAsync(r->x.data(), P.x, sizeof(double) * P.g.N, cudaMemcpyDeviceToHost, P.stream);
    cudaStreamSynchronize(P.stream);
    S.t_copy += std::chrono::duration<double>(Clock::now() - tc).count();
    r->t_done = S.now();
    r->state = r->info.status == IIM_OK ? kFinished : kFailed;
    r->error = (iim_status)r->info.status;
    free_problem(S, r, r->state == kFinished);
    S.note_fin.push_back(r->id);
  }
  // 4. requests the workers have created: check the exact size against the budget
  std::vector<Request*> got;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    got.swap(S.created);
  }
  for (Request* r : got) {
    --S.creating;
    S.in_use -= r->reserved;
    r->reserved = 0;
    S.in_use -= r->freed_bytes;          // a pooled problem given up by the worker
    r->freed_bytes = 0;
    if (r->reuse && r->create_status == IIM_OK) {
      // the reused problem's bytes have been counted all along
      r->reuse = false;
      r->state = kNeedData;
      S.note_need.push_back(r->id);
      continue;
    }
    if (r->create_status != IIM_OK) {
      r->state = kFailed;
      r->error = r->create_status;
      r->t_done = S.now();
      S.free_streams.push_back(r->stream);
      r->stream = nullptr;
      S.note_fin.push_back(r->id);
      continue;
    }
    r->bytes = r->prob->P.bytes;
    if (S.in_use + r->bytes > S.budget) {
      // larger than estimated and no room now: give the memory back and wait for room
      r->known_bytes = r->bytes;
      iim_problem_destroy(r->prob);
      r->prob = nullptr;
      S.free_streams.push_back(r->stream);
      r->stream = nullptr;
      if (r->known_bytes > S.budget) {
        r->state = kFailed;
        r->error = IIM_ERR_BUDGET;
        r->t_done = S.now();
        S.note_fin.push_back(r->id);
      } else {
        r->state = kQueued;
        S.queue.push_front(r);
      }
      continue;
    }
    S.in_use += r->bytes;
    S.peak = S.in_use > S.peak ? S.in_use : S.peak;
    r->state = kNeedData;
    S.note_need.push_back(r->id);
  }
  // requests cancelled while they were being created
  for (Request* r : got)
    if (r->cancel && (r->state == kNeedData || r->state == kQueued)) cancel_now(S, r);
  // 5. admission by budget, in submission order: reserve and hand to the workers
  while (!S.queue.empty()) {
    Request* r = S.queue.front();
    if (S.pooling && poolable(r->desc)) {
      // a retired problem of the same kind: no allocation, its set-up is re-run in place
      const PoolKey key = pool_key(r->desc);
      int best = -1;
      for (size_t k = 0; k < S.pool.size(); ++k)
        if (S.pool[k].key == key && (best < 0 || S.pool[k].stamp > S.pool[best].stamp)) best = (int)k;
      if (best >= 0) {
        PoolEntry e = S.pool[best];
        S.pool[best] = S.pool.back();
        S.pool.pop_back();
        S.queue.pop_front();
        r->prob = e.prob;
        r->stream = e.stream;
        r->bytes = e.bytes;
        r->reuse = true;
        r->reserved = 0;
        r->state = kCreating;
        ++S.creating;
        ++S.pool_hits;
        {
          std::lock_guard<std::mutex> lk(S.mu);
          S.to_create.push_back(r);
        }
        S.cv.notify_one();
        continue;
      }
    }
    const size_t need = r->known_bytes ? r->known_bytes : estimate_bytes(r->desc, S.opt);
    pool_evict(S, need);
    if (S.in_use + need > S.budget) break;
    S.queue.pop_front();
    ++S.pool_misses;
    if (!S.free_streams.empty()) {
      r->stream = S.free_streams.back();
      S.free_streams.pop_back();
    } else if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return IIM_ERR_CUDA;
    }
    r->reserved = need;
    S.in_use += need;
    r->state = kCreating;
    ++S.creating;
    {
      std::lock_guard<std::mutex> lk(S.mu);
      S.to_create.push_back(r);
    }
    S.cv.notify_one();
  }
  S.peak = S.in_use > S.peak ? S.in_use : S.peak;
  // report as many as the caller's arrays hold; the rest wait for the next step
  while (!S.note_need.empty() && need_data && nn < cap_need) {
    need_data[nn++] = S.note_need.front();
    S.note_need.pop_front();
  }
  while (!S.note_fin.empty() && finished && nf < cap_fin) {
    finished[nf++] = S.note_fin.front();
    S.note_fin.pop_front();
  }
  S.t_step += std::chrono::duration<double>(Clock::now() - t_enter).count();
  if (n_need) *n_need = nn;
  if (n_fin) *n_fin = nf;
  return IIM_OK;
}

iim_status iim_server_set_mode(iim_server* H, int mode) {
  if (!H || mode < 0 || mode > 1 || !H->S.reqs.empty()) return IIM_ERR_INVALID_ARG;
  H->S.mode = mode;
  return IIM_OK;
}

iim_problem* iim_server_problem(iim_server* H, int64_t id) {
  if (!H) return nullptr;
  auto it = H->S.reqs.find(id);
  if (it == H->S.reqs.end() || it->second->state != kNeedData) return nullptr;
  return it->second->prob;
}

iim_status iim_server_data_ready(iim_server* H, int64_t id) {
  if (!H) return IIM_ERR_INVALID_ARG;
  auto it = H->S.reqs.find(id);
  if (it == H->S.reqs.end() || it->second->state != kNeedData) return IIM_ERR_INVALID_ARG;
  // the data copies and the right-hand side have read the caller's buffers once this returns
  cudaStreamSynchronize(it->second->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("server data: ") + cudaGetErrorString(e));
    return IIM_ERR_CUDA;
  }
  it->second->state = kReady;
  return IIM_OK;
}

iim_status iim_server_cancel(iim_server* H, int64_t id) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Server& S = H->S;
  auto it = S.reqs.find(id);
  if (it == S.reqs.end()) return IIM_ERR_INVALID_ARG;
  Request* r = it->second;
  switch (r->state) {
    case kQueued:
    case kNeedData:
    case kReady:
      cancel_now(S, r);
      return IIM_OK;
    case kCreating:
    case kRunning:
    case kRetired:
      r->cancel = true;               // ends at the step that sees its creation or its solve end
      return IIM_OK;
    default:
      return IIM_ERR_INVALID_ARG;     // already finished or failed
  }
}

iim_status iim_server_take(iim_server* H, int64_t id, double* x_host, iim_solve_info* info, double* latency_s) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Server& S = H->S;
  auto it = S.reqs.find(id);
  if (it == S.reqs.end()) return IIM_ERR_INVALID_ARG;
  Request* r = it->second;
  if (r->state != kFinished && r->state != kFailed) return IIM_ERR_TIMEOUT;
  if (x_host && !r->x.empty()) std::memcpy(x_host, r->x.data(), sizeof(double) * r->x.size());
  if (info) *info = r->info;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  const iim_status st = r->state == kFinished ? IIM_OK : (r->error != IIM_OK ? r->error : IIM_ERR_NOT_CONVERGED);
  S.reqs.erase(it);
  delete r;
  return st;
}

iim_status iim_server_stats(iim_server* H, size_t* bytes_in_use, size_t* peak_bytes, int* queued, int* resident,
                            int64_t* runs, double* host_seconds, int* states) {
  if (!H) return IIM_ERR_INVALID_ARG;
  Server& S = H->S;
  if (host_seconds) {
    std::lock_guard<std::mutex> lk(S.mu);
    host_seconds[0] = S.t_step;
    host_seconds[1] = S.t_copy;
    host_seconds[2] = S.t_create;
  }
  if (bytes_in_use) *bytes_in_use = S.in_use;
  if (peak_bytes) *peak_bytes = S.peak;
  if (states) {
    for (int k = 0; k < 8; ++k) states[k] = 0;
    for (auto& kv : S.reqs) ++states[kv.second->state];
  }
  if (queued) *queued = (int)S.queue.size();
  if (resident) *resident = S.resident;
  if (runs) *runs = S.runs;
  return IIM_OK;
}

}  // extern "C"
