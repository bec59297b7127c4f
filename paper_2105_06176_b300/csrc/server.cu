// Continuous-batching solve server (ppcg_server_* in include/ppcg.h).
//
// Three host threads share one device:
//   admitters -- one for requests the cluster path takes (up to cluster_max_rows rows), one
//                for larger ones; each takes its class's queued requests in arrival order
//                while their device footprint fits in the HBM budget (an older request of
//                the other class that is waiting for memory keeps its turn), builds the
//                handle (CSR -> SELL on the device) on its own stream, stages b and x0, and
//                hands the resident solve to the executor, so a small request is never
//                queued behind the matrix conversion of a large one;
//   executor  -- runs epochs: every resident CLUSTER-path solve (up to 131,072 rows)
//                advances inside one persistent cluster launch by its own budget,
//                epoch_iters * 131072 / n iterations (clamped to [2, 64 epoch_iters]), so
//                each gets about the same device time and their work overlaps; GRID-path
//                solves run in arrival order, the two oldest getting a whole-GPU slice of
//                clamp(2.5e8 / n, 32, 4000) iterations (2.5e8 row-iterations, about 5-10
//                ms) per epoch; finished solves are copied out, their memory released, and
//                requests that arrived meanwhile join at the next epoch.
// A solve's vectors, scalars and control block stay on the device between epochs, and its
// partition over CTAs depends only on its handle, so a result is bitwise the same alone or
// in any mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "handle.h"

namespace {

using namespace ppcg;

constexpr size_t kMaxQueue = 1 << 20;

struct Request {
  uint64_t ticket = 0;
  int64_t n = 0, nnz = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> col;
  std::vector<double> val, b, x0;
  bool has_x0 = false;
  double tol = 0.0;
  int32_t maxit = 0;
  size_t footprint = 0;
};

struct Slot {
  uint64_t ticket = 0;
  ppcg_handle h = nullptr;
  size_t footprint = 0;
};

struct Result {
  int32_t status = PPCG_OK;
  std::vector<double> x;
  ppcg_info info;
};

}  // namespace

struct ppcg_srv {
  int device = 0;
  ppcg_opts opts;
  size_t budget = 0;
  int epoch_iters = 256;
  std::mutex mu;
  std::condition_variable cv_admit, cv_exec;
  std::deque<std::unique_ptr<Request>> queue;
  std::vector<Slot> ready;
  std::unordered_map<uint64_t, Result> done;
  std::unordered_set<uint64_t> live;   // queued or running
  size_t in_use = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  int64_t completed = 0, running = 0;
  std::thread admitter[2], executor;
  cudaStream_t s_admit[2] = {nullptr, nullptr}, s_exec = nullptr;
  // executor scratch for cluster epochs
  SysDesc* d_descs = nullptr;
  int32_t* d_lists = nullptr;
  size_t cap = 0;
};

namespace {

void finish(ppcg_srv* S, uint64_t ticket, Result&& r) {
  std::lock_guard<std::mutex> lk(S->mu);
  S->done[ticket] = std::move(r);
  S->live.erase(ticket);
  S->completed++;
}

// Admission class of a request: 0 = the cluster path's sizes, 1 = larger.
int admit_class(const ppcg_srv* S, const Request& r) { return r.n <= S->opts.cluster_max_rows ? 0 : 1; }

// Index of the request admitter `cls` may take now, or -1: the oldest queued request of its
// class, if it fits the budget and no older request (of the other class) is waiting for
// memory.  Called with S->mu held.
long next_admissible(const ppcg_srv* S, int cls) {
  for (size_t i = 0; i < S->queue.size(); i++) {
    const Request& r = *S->queue[i];
    const bool fits = S->in_use + r.footprint <= S->budget;
    if (admit_class(S, r) == cls) return fits ? (long)i : -1;
    if (!fits) return -1;
  }
  return -1;
}

void admit_loop(ppcg_srv* S, int cls) {
  cudaSetDevice(S->device);
  cudaStream_t stream = S->s_admit[cls];
  for (;;) {
    std::unique_ptr<Request> req;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      long idx = -1;
      S->cv_admit.wait(lk, [&] { return S->stop || (idx = next_admissible(S, cls)) >= 0; });
      if (S->stop) return;
      req = std::move(S->queue[(size_t)idx]);
      S->queue.erase(S->queue.begin() + idx);
      S->in_use += req->footprint;
      S->running++;
    }
    NvtxRange nvtx_range("ppcg_server_admit");
    ppcg_handle h = nullptr;
    // Served solves take the cluster path (epochs of many solves in one launch) or the grid
    // path; the on-chip path holds 8 SMs' shared memory per solve and is left to ppcg_solve.
    ppcg_opts o = S->opts;
    if (o.path == PPCG_PATH_AUTO || o.path == PPCG_PATH_ONCHIP)
      o.path = req->n <= o.cluster_max_rows ? PPCG_PATH_CLUSTER : PPCG_PATH_GRID;
    // one cluster size for every served solve: an epoch is one launch of clusters
    o.cluster_ctas = kClusterSize;
    ppcg_status st = ppcg_create(&h, req->n, req->nnz, req->rp.data(), req->col.data(), req->val.data(), &o,
                                 stream);
    Slot slot;
    slot.ticket = req->ticket;
    slot.footprint = req->footprint;
    if (st == PPCG_OK && req->n > 0) {
      slot.h = h;
      st = stage_inputs(h, req->b.data(), req->has_x0 ? req->x0.data() : nullptr, false, stream);
      if (st == PPCG_OK) {
        prepare_control(h, req->tol, req->maxit, stream);
        cudaMemcpyAsync(h->d_desc, &h->desc, sizeof(SysDesc), cudaMemcpyHostToDevice, stream);
        if (cudaStreamSynchronize(stream) != cudaSuccess) { cudaGetLastError(); st = PPCG_ERR_CUDA; }
      }
    }
    if (st != PPCG_OK || req->n == 0) {
      Result r;
      memset(&r.info, 0, sizeof(r.info));
      r.status = st;
      r.info.status = st;
      if (h) ppcg_destroy(h);
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->in_use -= req->footprint;
        S->running--;
      }
      finish(S, req->ticket, std::move(r));
      S->cv_admit.notify_all();
      continue;
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->ready.push_back(slot);
    }
    S->cv_exec.notify_all();
  }
}

bool run_cluster_epoch(ppcg_srv* S, const std::vector<Slot*>& slots) {
  NvtxRange nvtx_range("ppcg_server_epoch");
  const int m = (int)slots.size();
  if (m == 0) return true;
  std::vector<SysDesc> descs(m);
  std::vector<double> cost(m);
  for (int k = 0; k < m; k++) {
    descs[k] = slots[k]->h->desc;
    // Same work per solve and epoch: epoch_iters iterations for a 2^17-row system, more for
    // smaller ones (at most 64x), fewer for larger ones (at least 2).
    const double n = (double)std::max<int64_t>(slots[k]->h->n, 1);
    const double it = std::min(64.0 * S->epoch_iters, std::max(2.0, S->epoch_iters * 131072.0 / n));
    descs[k].budget = (int32_t)it;
    cost[k] = cluster_solve_cost(slots[k]->h, it);
  }
  // Longest first: a static longest-processing-time assignment while there are at most two
  // solves per cluster, else the clusters take solves from a shared counter (as in
  // ppcg_batch_solve).
  const int nclusters = std::max(1, std::min(m, max_active_clusters(S->device, kClusterSize)));
  std::vector<int32_t> order(m);
  for (int k = 0; k < m; k++) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  const bool dynamic = m > 2 * nclusters;
  std::vector<int32_t> packed;   // dynamic: order, counter; static: list_ptr, lists
  if (dynamic) {
    packed = order;
    packed.push_back(0);
  } else {
    std::vector<std::vector<int>> lists(nclusters);
    std::vector<double> load(nclusters, 0.0);
    for (int k : order) {
      const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lists[c].push_back(k);
      load[c] += cost[k];
    }
    packed.push_back(0);
    for (auto& l : lists) packed.push_back(packed.back() + (int32_t)l.size());
    for (auto& l : lists) packed.insert(packed.end(), l.begin(), l.end());
  }
  if ((size_t)m > S->cap || packed.size() > 2 * S->cap + 2) {
    cudaFree(S->d_descs);
    cudaFree(S->d_lists);
    S->cap = std::max<size_t>(2 * (size_t)m, 64);
    if (cudaMalloc(&S->d_descs, S->cap * sizeof(SysDesc)) != cudaSuccess ||
        cudaMalloc(&S->d_lists, (2 * S->cap + 2) * sizeof(int32_t)) != cudaSuccess) {
      cudaGetLastError();
      S->cap = 0;
      return false;
    }
  }
  cudaMemcpyAsync(S->d_descs, descs.data(), m * sizeof(SysDesc), cudaMemcpyHostToDevice, S->s_exec);
  cudaMemcpyAsync(S->d_lists, packed.data(), packed.size() * sizeof(int32_t), cudaMemcpyHostToDevice, S->s_exec);
  const cudaError_t e =
      dynamic ? launch_clusters(S->d_descs, S->d_lists, nullptr, nclusters, S->epoch_iters, S->s_exec, false,
                                S->d_lists + m, m)
              : launch_clusters(S->d_descs, S->d_lists + nclusters + 1, S->d_lists, nclusters, S->epoch_iters,
                                S->s_exec);
  return e == cudaSuccess;
}

void exec_loop(ppcg_srv* S) {
  cudaSetDevice(S->device);
  std::vector<Slot> active;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_exec.wait(lk, [&] { return S->stop || !S->ready.empty() || !active.empty(); });
      if (S->stop) break;
      for (Slot& s : S->ready) active.push_back(s);
      S->ready.clear();
    }
    std::vector<Slot*> cl, gr;
    for (Slot& s : active) (s.h->path == PPCG_PATH_CLUSTER ? cl : gr).push_back(&s);
    bool ok = run_cluster_epoch(S, cl);
    // Whole-GPU solves in arrival order: the two oldest each get a slice of 2.5e8
    // row-iterations (about 5-10 ms of streaming work); later ones wait.  Slices four times
    // as long left the large requests' p99 where it was (their own solve time sets it) and
    // doubled the small requests' median.
    for (size_t k = 0; k < gr.size() && k < 2; k++) {
      Slot* s = gr[k];
      const double n = (double)std::max<int64_t>(s->h->n, 1);
      const int slice = (int)std::min(4000.0, std::max(32.0, 2.5e8 / n));
      cudaMemsetAsync(s->h->bar, 0, sizeof(unsigned), S->s_exec);
      ok = ok && launch_grid(s->h->d_desc, s->h->shape, s->h->grid, slice, S->s_exec) == cudaSuccess;
    }
    for (Slot& s : active) {
      cudaMemcpyAsync(&s.h->stage->ctl, s.h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, S->s_exec);
      cudaMemcpyAsync(&s.h->stage->err, s.h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, S->s_exec);
    }
    if (cudaStreamSynchronize(S->s_exec) != cudaSuccess || !ok) {
      cudaGetLastError();
      // fail every resident solve rather than spin on a broken stream
      for (Slot& s : active) { s.h->stage->ctl.state = S_DONE; s.h->stage->ctl.status = PPCG_ERR_CUDA; }
    }
    std::vector<Slot> keep;
    for (Slot& s : active) {
      const Stage& sg = *s.h->stage;
      if (sg.ctl.state != S_DONE && sg.err == 0) { keep.push_back(s); continue; }
      Result r;
      r.x.resize(s.h->n);
      s.h->stream = S->s_exec;
      stage_outputs(s.h, r.x.data(), S->s_exec);
      cudaStreamSynchronize(S->s_exec);
      InfoJob j{s.h->stage, &r.info, s.h->bytes_per_iter, s.h->opts.norm, s.h->opts.precision};
      fill_info(sg, j, &r.info);
      r.status = r.info.status;
      ppcg_destroy(s.h);
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->in_use -= s.footprint;
        S->running--;
      }
      finish(S, s.ticket, std::move(r));
      S->cv_admit.notify_all();
    }
    active.swap(keep);
  }
  for (Slot& s : active) ppcg_destroy(s.h);
}

}  // namespace

extern "C" {

ppcg_status ppcg_server_create(ppcg_server* server, size_t hbm_budget, const ppcg_opts* opts) {
  if (!server) { set_error("ppcg_server_create: NULL"); return PPCG_ERR_ARG; }
  *server = nullptr;
  ppcg_srv* S = new ppcg_srv();
  ppcg_opts_default(&S->opts);
  if (opts) S->opts = *opts;
  // Default plan: requests up to 131,072 rows run on thread-block clusters (all of them
  // advance together inside one launch per epoch); larger ones use the whole GPU.
  if (S->opts.path == PPCG_PATH_AUTO && (!opts || opts->cluster_max_rows == 16384)) S->opts.cluster_max_rows = 131072;
  if (S->opts.epoch_iters > 0) S->epoch_iters = S->opts.epoch_iters;
  cudaGetDevice(&S->device);
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    set_error("ppcg_server_create: no CUDA device");
    return PPCG_ERR_CUDA;
  }
  S->budget = hbm_budget ? hbm_budget : (size_t)(0.9 * (double)fr);
  if (cudaStreamCreateWithFlags(&S->s_admit[0], cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->s_admit[1], cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->s_exec, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    set_error("ppcg_server_create: stream creation failed");
    return PPCG_ERR_CUDA;
  }
  S->admitter[0] = std::thread(admit_loop, S, 0);
  S->admitter[1] = std::thread(admit_loop, S, 1);
  S->executor = std::thread(exec_loop, S);
  *server = S;
  return PPCG_OK;
}

ppcg_status ppcg_submit(ppcg_server S, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                        const double* val, const double* b, const double* x0, double tol, int32_t maxit,
                        uint64_t* ticket) {
  if (!S || !ticket || n < 0 || nnz < 0 || !(tol >= 0.0) || maxit < 0 ||
      (n > 0 && (!row_ptr || !col || !val || !b))) {
    set_error("ppcg_submit: bad arguments");
    return PPCG_ERR_ARG;
  }
  auto req = std::make_unique<Request>();
  req->n = n;
  req->nnz = nnz;
  req->rp.assign(row_ptr, row_ptr + (n + 1));
  req->col.assign(col, col + nnz);
  req->val.assign(val, val + nnz);
  req->b.assign(b, b + n);
  if (x0) { req->x0.assign(x0, x0 + n); req->has_x0 = true; }
  req->tol = tol;
  req->maxit = maxit;
  req->footprint = footprint_bytes(n, nnz, S->opts.precision);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (req->footprint > S->budget) { set_error("ppcg_submit: request larger than the HBM budget"); return PPCG_ERR_OOM; }
    if (S->queue.size() >= kMaxQueue) { set_error("ppcg_submit: queue full"); return PPCG_ERR_BUSY; }
    req->ticket = S->next_ticket++;
    *ticket = req->ticket;
    S->live.insert(req->ticket);
    S->queue.push_back(std::move(req));
  }
  S->cv_admit.notify_all();
  return PPCG_OK;
}

ppcg_status ppcg_poll(ppcg_server S, uint64_t ticket, double* x_out, ppcg_info* info) {
  if (!S) { set_error("ppcg_poll: NULL server"); return PPCG_ERR_ARG; }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->done.find(ticket);
  if (it == S->done.end()) {
    if (S->live.count(ticket)) return PPCG_PENDING;
    set_error("ppcg_poll: unknown ticket %llu", (unsigned long long)ticket);
    return PPCG_ERR_UNKNOWN_TICKET;
  }
  Result& r = it->second;
  if (x_out && !r.x.empty()) memcpy(x_out, r.x.data(), r.x.size() * sizeof(double));
  if (info) *info = r.info;
  ppcg_status st = (ppcg_status)r.status;
  S->done.erase(it);
  return st;
}

ppcg_status ppcg_server_stats(ppcg_server S, int64_t* completed, int64_t* running, int64_t* queued,
                              int64_t* hbm_in_use) {
  if (!S) { set_error("ppcg_server_stats: NULL server"); return PPCG_ERR_ARG; }
  std::lock_guard<std::mutex> lk(S->mu);
  if (completed) *completed = S->completed;
  if (running) *running = S->running;
  if (queued) *queued = (int64_t)S->queue.size();
  if (hbm_in_use) *hbm_in_use = (int64_t)S->in_use;
  return PPCG_OK;
}

void ppcg_server_destroy(ppcg_server S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_admit.notify_all();
  S->cv_exec.notify_all();
  for (std::thread& t : S->admitter)
    if (t.joinable()) t.join();
  if (S->executor.joinable()) S->executor.join();
  for (Slot& s : S->ready) ppcg_destroy(s.h);
  cudaFree(S->d_descs);
  cudaFree(S->d_lists);
  cudaStreamDestroy(S->s_admit[0]);
  cudaStreamDestroy(S->s_admit[1]);
  cudaStreamDestroy(S->s_exec);
  delete S;
}

}  // extern "C"
