// C ABI of the solver (include/ppcg.h): handles, solve, batch solve.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "handle.h"

namespace ppcg {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {nullptr};
std::vector<Stage*> g_stage_free;     // pinned info stages, reused across handles
}  // namespace

// Host-side fault injection for tests: with PPCG_FAIL_DEVICE_ALLOC=k set, the k-th device
// allocation counted from the moment the variable took its current value fails as out of
// memory (once).  No GPU fault is involved: the allocation is simply not made.
static bool injected_alloc_failure() {
  static std::mutex mu;
  static std::string last;
  static long count = 0;
  const char* e = getenv("PPCG_FAIL_DEVICE_ALLOC");
  std::lock_guard<std::mutex> lk(mu);
  if (!e || !*e) { last.clear(); return false; }
  if (last != e) { last = e; count = 0; }
  const long k = atol(e);
  return k > 0 && ++count == k;
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st) {
  if (injected_alloc_failure()) { *p = nullptr; return cudaErrorMemoryAllocation; }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev >= 0 && dev < 64 && !g_pools[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      if (cudaMemPoolCreate(&g_pools[dev], &props) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
      } else {
        cudaGetLastError();
        g_pools[dev] = nullptr;
      }
    }
    if (dev >= 0 && dev < 64) pool = g_pools[dev];
  }
  cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

void pool_free(void* p, cudaStream_t st) {
  if (p && cudaFreeAsync(p, st) != cudaSuccess) cudaGetLastError();
}

static Stage* stage_get() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_stage_free.empty()) {
    Stage* blk = nullptr;
    if (cudaMallocHost((void**)&blk, 64 * sizeof(Stage)) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    for (int i = 0; i < 64; i++) g_stage_free.push_back(blk + i);
  }
  Stage* s = g_stage_free.back();
  g_stage_free.pop_back();
  memset(s, 0, sizeof(Stage));
  return s;
}

static void stage_put(Stage* s) {
  if (!s) return;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  g_stage_free.push_back(s);
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

namespace {

__global__ void k_gather(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ src,
                         double* __restrict__ dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[perm[i]];
}

// Slot `slot` of a chunk-interleaved block with ns slots: element i at
// (i / 32) * ns * 32 + slot * 32 + i % 32.
__host__ __device__ __forceinline__ int64_t slot_index(int64_t i, int ns, int slot) {
  return (i >> 5) * (int64_t)ns * kChunk + (int64_t)slot * kChunk + (i & 31);
}

// plain vector (optionally read through the row permutation) -> block slot
template <typename T>
__global__ void k_to_slot(int64_t n, const int32_t* __restrict__ perm, const T* __restrict__ src,
                          T* __restrict__ blk, int ns, int slot) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) blk[slot_index(i, ns, slot)] = src[perm ? perm[i] : i];
}

// plain -> block slot divided by the scale slot (x~ = x / sig), optional row permutation
__global__ void k_to_slot_unscale(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ src,
                                  double* __restrict__ blk, int ns, int slot, int sig_slot) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) blk[slot_index(i, ns, slot)] = src[perm ? perm[i] : i] / blk[slot_index(i, ns, sig_slot)];
}

// block slot times the scale slot -> plain (x = sig * x~), optional row permutation
__global__ void k_from_slot_scale(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ blk,
                                  int ns, int slot, int sig_slot, double* __restrict__ dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[perm ? perm[i] : i] = blk[slot_index(i, ns, slot)] * blk[slot_index(i, ns, sig_slot)];
}

// d and sig = d^-1/2 slots of the Jacobi-scaled block
__global__ void k_fill_scale_slots(int64_t n, const double* __restrict__ diag, double* __restrict__ blk, int ns,
                                   int dslot, int sslot) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const double d = diag[i];
    blk[slot_index(i, ns, dslot)] = d;
    blk[slot_index(i, ns, sslot)] = 1.0 / sqrt(d);
  }
}

__global__ void k_fill_slot(int64_t n, double* __restrict__ blk, int ns, int slot, double v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) blk[slot_index(i, ns, slot)] = v;
}

// block slot -> plain vector (optionally written through the row permutation)
__global__ void k_from_slot(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ blk, int ns,
                            int slot, double* __restrict__ dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[perm ? perm[i] : i] = blk[slot_index(i, ns, slot)];
}

__global__ void k_fill_plain(int64_t n, double* __restrict__ p, double v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_init_ctl(Ctl* c, int32_t state) {
  Ctl z;
  memset(&z, 0, sizeof(z));
  z.state = state;
  z.last_rr_iter = -1;
  z.status = PPCG_ERR_NOT_CONVERGED;
  *c = z;
}

unsigned blocks_for(int64_t n, int tb) { return (unsigned)((n + tb - 1) / tb); }

void CUDART_CB info_callback(void* p) {
  std::vector<InfoJob>* jobs = static_cast<std::vector<InfoJob>*>(p);
  for (const InfoJob& j : *jobs)
    if (j.info) fill_info(*j.stage, j, j.info);
  delete jobs;
}

}  // namespace

template <typename T>
static bool walloc(ppcg_ctx* h, T** p, size_t count) {
  if (pool_alloc((void**)p, std::max<size_t>(count, 1) * sizeof(T), h->stream) != cudaSuccess) return false;
  h->allocs.push_back(*p);
  return true;
}

// Releases a handle's memory in the order of its last stream (after its last solve).
static void free_all(ppcg_ctx* h) {
  for (void* p : h->allocs) pool_free(p, h->stream);
  h->allocs.clear();
  stage_put(h->stage);
  h->stage = nullptr;
}

// Enqueue: b/x0 -> solver-order device vectors; fills h->desc pointers for this solve.
// Returns the device x the solver writes (user x itself when possible).
ppcg_status stage_inputs(ppcg_ctx* h, const double* b, const double* x0, bool require_device, cudaStream_t st) {
  const int64_t n = h->n;
  const size_t bytes = n * sizeof(double);
  const bool bd = is_device_ptr(b);
  const bool x0d = x0 ? is_device_ptr(x0) : true;
  if (require_device && (!bd || !x0d)) {
    set_error("ppcg_batch_solve: b, x0 and x must be device pointers");
    return PPCG_ERR_ARG;
  }
  // b: used in place when it is a device vector in solver order, else staged into b_ws
  const double* bsol;
  if (h->perm) {
    const double* src = b;
    if (!bd) { cudaMemcpyAsync(h->tmp, b, bytes, cudaMemcpyHostToDevice, st); src = h->tmp; }
    k_gather<<<blocks_for(n, 256), 256, 0, st>>>(n, h->perm, src, h->b_ws);
    bsol = h->b_ws;
  } else if (bd) {
    bsol = b;
  } else {
    cudaMemcpyAsync(h->b_ws, b, bytes, cudaMemcpyHostToDevice, st);
    bsol = h->b_ws;
  }
  // x0 -> the x slot of the vector block, in solver row order
  int32_t x_zero = 0;
  if (!x0) {
    k_fill_slot<<<blocks_for(n, 256), 256, 0, st>>>(n, h->desc.v64, h->ns64, h->xslot, 0.0);
    x_zero = 1;
  } else {
    const double* src = x0;
    if (!x0d) { cudaMemcpyAsync(h->tmp, x0, bytes, cudaMemcpyHostToDevice, st); src = h->tmp; }
    if (h->opts.variant == PPCG_VARIANT_JACOBI_SCALED)
      k_to_slot_unscale<<<blocks_for(n, 256), 256, 0, st>>>(n, h->perm, src, h->desc.v64, h->ns64, h->xslot, kSlotSigS);
    else
      k_to_slot<double><<<blocks_for(n, 256), 256, 0, st>>>(n, h->perm, src, h->desc.v64, h->ns64, h->xslot);
  }
  h->desc.b = bsol;
  h->desc.x_zero = x_zero;
  return PPCG_OK;
}

void stage_outputs(ppcg_ctx* h, double* x, cudaStream_t st) {
  const int64_t n = h->n;
  const bool xd = is_device_ptr(x);
  if (h->opts.variant == PPCG_VARIANT_JACOBI_SCALED)
    k_from_slot_scale<<<blocks_for(n, 256), 256, 0, st>>>(n, h->perm, h->desc.v64, h->ns64, h->xslot, kSlotSigS,
                                                          xd ? x : h->tmp);
  else
    k_from_slot<<<blocks_for(n, 256), 256, 0, st>>>(n, h->perm, h->desc.v64, h->ns64, h->xslot, xd ? x : h->tmp);
  if (!xd) cudaMemcpyAsync(x, h->tmp, n * sizeof(double), cudaMemcpyDeviceToHost, st);
}

void prepare_control(ppcg_ctx* h, double tol, int32_t maxit, cudaStream_t st) {
  h->desc.tol = tol;
  h->desc.maxit = maxit;
  k_init_ctl<<<1, 1, 0, st>>>(h->ctl, h->opts.precision == PPCG_FP32_IR   ? S_O_START
                                      : h->opts.precision == PPCG_FP32_RU ? S_U_START
                                                                          : S_START);
  cudaMemsetAsync(h->bar, 0, sizeof(unsigned), st);
  cudaMemsetAsync(h->err, 0, sizeof(int32_t), st);
}

size_t footprint_bytes(int64_t n, int64_t nnz, int32_t precision) {
  const bool fp32 = precision != PPCG_FP64;
  const double slots = 1.05 * (double)nnz + 32.0 * ((double)n / 32.0 + 1.0);
  // matrix (values, columns and the one-byte column dictionary) + cptr/diag/invd/b/tmp/perm
  double bytes = slots * (fp32 ? 17.0 : 13.0) + (double)n * 8.0 * 6.0;
  bytes += (double)n * 8.0 * 10.0 + (fp32 ? (double)n * 4.0 * 11.0 : 0.0);
  return (size_t)bytes + (1u << 20);
}

namespace {

// Work list of a launch of one cluster running system 0: device array {0, 0, 1} read as
// list = {0} (element 0) and list_ptr = {0, 1} (elements 1-2).
// (One array per device, created on first use and kept for the process.)
const int32_t* single_work_list() {
  static std::mutex mu;
  static std::unordered_map<int, int32_t*> per;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  int32_t*& d_list = per[dev];
  if (!d_list) {
    const int32_t host[3] = {0, 0, 1};
    if (cudaMalloc(&d_list, sizeof(host)) != cudaSuccess ||
        cudaMemcpy(d_list, host, sizeof(host), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      d_list = nullptr;
    }
  }
  return d_list;
}

// Cluster size of a CLUSTER-path plan (opts.cluster_ctas == 0).  In a batch the GPU is
// shared by many clusters, so what a system costs is the CTA-time of an iteration: its
// time per iteration on a cluster of cs CTAs times cs.  Small systems are bound by the
// per-iteration barrier, reduction and control step, which a few CTAs do as fast as many
// (small clusters win); large ones by their bytes, which more CTAs move proportionally
// faster (the size barely changes the cost, and the larger size shortens the batch's
// tail).  So each candidate of {2, 4, 8} is timed on the device -- the handle's own
// system, b = 1, x0 = 0, the difference of a 4- and a 24-iteration run of one cluster --
// and the largest size within 10% of the least CTA-time wins.  (16-CTA clusters lost in
// every batch measured: fewer clusters, and a second launch for the rest.)  The choice is
// cached per device, precision, variant, norm, offset pattern, nonzeros per row and
// half-octave of rows, so a family of similar systems is timed once.
int tune_cluster_size(ppcg_ctx* h, cudaStream_t st) {
  static std::mutex mu;
  static std::map<std::array<int64_t, 7>, int> cache;
  const int64_t n = h->n;
  const std::array<int64_t, 7> key{h->device, h->opts.precision, h->opts.variant, h->opts.norm, h->A.pat_k,
                                   std::llround(2.0 * (double)h->nnz / (double)n),
                                   std::llround(2.0 * std::log2((double)n))};
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  const int32_t* list = single_work_list();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!list || cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return kClusterSize;
  }
  k_fill_plain<<<blocks_for(n, 256), 256, 0, st>>>(n, h->b_ws, 1.0);
  const double* b_keep = h->desc.b;
  const int32_t xz_keep = h->desc.x_zero;
  h->desc.b = h->b_ws;
  auto run = [&](int cs, int iters, float* ms) -> bool {
    k_fill_slot<<<blocks_for(n, 256), 256, 0, st>>>(n, h->desc.v64, h->ns64, h->xslot, 0.0);
    h->desc.x_zero = 1;
    prepare_control(h, 0.0, iters, st);
    cudaMemcpyAsync(h->d_desc, &h->desc, sizeof(SysDesc), cudaMemcpyHostToDevice, st);
    cudaEventRecord(e0, st);
    if (launch_clusters(h->d_desc, list, list + 1, 1, 0, st, false, nullptr, 0, cs) != cudaSuccess) return false;
    cudaEventRecord(e1, st);
    return cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(ms, e0, e1) == cudaSuccess;
  };
  double cost[3] = {0, 0, 0};
  const int cands[3] = {2, 4, 8};
  double best = HUGE_VAL;
  for (int k = 0; k < 3; k++) {
    cost[k] = HUGE_VAL;
    if (max_active_clusters(h->device, cands[k]) < 1) continue;
    float warm = 0.f, t4 = 0.f, t24 = 0.f;
    if (!run(cands[k], 2, &warm) || !run(cands[k], 4, &t4) || !run(cands[k], 24, &t24)) { cudaGetLastError(); continue; }
    cost[k] = std::max(1e-6, (double)(t24 - t4) / 20.0) * cands[k];
    best = std::min(best, cost[k]);
  }
  int cs = kClusterSize;
  if (best < HUGE_VAL)
    for (int k = 0; k < 3; k++)
      if (cost[k] <= 1.1 * best) cs = cands[k];
  h->desc.b = b_keep;
  h->desc.x_zero = xz_keep;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = cs;
  return cs;
}

// Side streams with a fork/join event pair each, per device (batch launches of the on-chip
// path, index 0, and of the cluster sizes after the first, indices 1-3, run beside the
// caller's stream).  Created on first use, kept for the process.
bool side_stream(int device, cudaStream_t* s, cudaEvent_t* fork, cudaEvent_t* join, int idx = 0) {
  struct Side { cudaStream_t s = nullptr; cudaEvent_t fork = nullptr, join = nullptr; };
  static std::mutex mu;
  static std::unordered_map<int, Side> per;
  std::lock_guard<std::mutex> lk(mu);
  Side& x = per[device * 8 + idx];
  if (!x.s) {
    if (cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      x = Side();
      return false;
    }
  }
  *s = x.s;
  *fork = x.fork;
  *join = x.join;
  return true;
}

// The solve's record (control block and launch error flag) into the handle's pinned stage.
void enqueue_stage_copies(ppcg_ctx* h, cudaStream_t st) {
  cudaMemcpyAsync(&h->stage->ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&h->stage->err, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  h->last_solve = 1;
}

void enqueue_info(std::vector<std::pair<ppcg_ctx*, ppcg_info*>>& items, cudaStream_t st) {
  auto* jobs = new std::vector<InfoJob>();
  for (auto& it : items) {
    ppcg_ctx* h = it.first;
    enqueue_stage_copies(h, st);
    jobs->push_back({h->stage, it.second, h->bytes_per_iter, h->opts.norm, h->opts.precision});
  }
  if (cudaLaunchHostFunc(st, info_callback, jobs) != cudaSuccess) {
    cudaGetLastError();
    delete jobs;
  }
}

bool check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return false;
  }
  return true;
}

void write_trivial_info(ppcg_info* info, int32_t status) {
  if (!info) return;
  memset(info, 0, sizeof(*info));
  info->status = status;
}

}  // namespace
}  // namespace ppcg

using namespace ppcg;

extern "C" {

void ppcg_opts_default(ppcg_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = PPCG_FP64;
  o->format = PPCG_FMT_AUTO;
  o->norm = PPCG_NORM_REL_R;
  o->path = PPCG_PATH_AUTO;
  o->sigma = 0;
  o->rr_period = 0;
  o->inner_tol = 1e-2;
  o->inner_maxit = 2000;
  o->max_outer = 100;
  o->spin_limit_ns = 10000000000LL;
  o->cluster_max_rows = 16384;
  o->epoch_iters = 256;
  o->max_restarts = 8;
  o->gap_theta = 1e-6;
  o->gap_fall = 100;
  o->cluster_ctas = 8;
}

const char* ppcg_last_error(void) { return g_err; }

ppcg_status ppcg_create(ppcg_handle* handle, int64_t n, int64_t nnz, const int64_t* row_ptr,
                        const int32_t* col, const double* val, const ppcg_opts* opts,
                        cudaStream_t stream) {
  NvtxRange nvtx_range("ppcg_create");
  const auto t_create = std::chrono::steady_clock::now();
  g_err[0] = 0;
  if (!handle) { set_error("ppcg_create: handle is NULL"); return PPCG_ERR_ARG; }
  *handle = nullptr;
  if (n < 0 || nnz < 0 || n > INT32_MAX || (n > 0 && (!row_ptr || !col || !val || nnz < n))) {
    set_error("ppcg_create: bad sizes or NULL arrays (n=%lld nnz=%lld)", (long long)n, (long long)nnz);
    return PPCG_ERR_ARG;
  }
  ppcg_ctx* h = new ppcg_ctx();
  ppcg_opts_default(&h->opts);
  if (opts) h->opts = *opts;
  if (h->opts.precision != PPCG_FP64 && h->opts.precision != PPCG_FP32_IR && h->opts.precision != PPCG_FP32_RU) {
    delete h; set_error("ppcg_create: bad precision"); return PPCG_ERR_ARG;
  }
  if (h->opts.precision == PPCG_FP32_RU && h->opts.norm != PPCG_NORM_REL_R) {
    delete h; set_error("ppcg_create: FP32_RU stops on the relative FP64 residual (norm REL_R only)"); return PPCG_ERR_ARG;
  }
  if (h->opts.norm != PPCG_NORM_REL_R && h->opts.norm != PPCG_NORM_PAPER_U_ABS) { delete h; set_error("ppcg_create: bad norm"); return PPCG_ERR_ARG; }
  if (h->opts.format < PPCG_FMT_AUTO || h->opts.format > PPCG_FMT_BOX) { delete h; set_error("ppcg_create: bad format"); return PPCG_ERR_ARG; }
  if (h->opts.variant != PPCG_VARIANT_ALG2 && h->opts.variant != PPCG_VARIANT_JACOBI_SCALED) {
    delete h; set_error("ppcg_create: bad variant"); return PPCG_ERR_ARG;
  }
  if (h->opts.variant == PPCG_VARIANT_JACOBI_SCALED && h->opts.precision != PPCG_FP64) {
    delete h; set_error("ppcg_create: the Jacobi-scaled variant is FP64 only"); return PPCG_ERR_ARG;
  }
  if (h->opts.spin_limit_ns <= 0) h->opts.spin_limit_ns = 10000000000LL;
  if (h->opts.inner_maxit <= 0) h->opts.inner_maxit = 2000;
  if (h->opts.max_outer <= 0) h->opts.max_outer = 100;
  if (!(h->opts.inner_tol > 0.0 && h->opts.inner_tol < 1.0)) h->opts.inner_tol = 1e-2;
  cudaGetDevice(&h->device);
  h->n = n;
  h->nnz = nnz;
  memset(&h->A, 0, sizeof(h->A));
  memset(&h->desc, 0, sizeof(h->desc));
  if (n == 0) { *handle = h; return PPCG_OK; }

  // Bring the CSR to the device (temporary copies when it lives on the host).
  std::vector<void*> tmp;
  h->stream = stream;
  auto free_tmp = [&]() { for (void* p : tmp) pool_free(p, stream); tmp.clear(); };
  const int64_t* d_rp = row_ptr;
  const int32_t* d_col = col;
  const double* d_val = val;
  auto upload = [&](const void* src, size_t bytes, const void** dst) -> bool {
    if (is_device_ptr(src)) { *dst = src; return true; }
    void* p = nullptr;
    if (pool_alloc(&p, std::max<size_t>(bytes, 1), stream) != cudaSuccess) return false;
    tmp.push_back(p);
    if (cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, stream) != cudaSuccess) { cudaGetLastError(); return false; }
    *dst = p;
    return true;
  };
  if (!upload(row_ptr, (n + 1) * sizeof(int64_t), (const void**)&d_rp) ||
      !upload(col, nnz * sizeof(int32_t), (const void**)&d_col) ||
      !upload(val, nnz * sizeof(double), (const void**)&d_val)) {
    free_tmp();
    delete h;
    set_error("ppcg_create: could not stage the CSR arrays on the device");
    return PPCG_ERR_OOM;
  }
  const bool want_box = h->opts.format == PPCG_FMT_AUTO || h->opts.format == PPCG_FMT_BOX;
  int32_t sigma = h->opts.format == PPCG_FMT_CSR || h->opts.format == PPCG_FMT_BOX ? 1 : h->opts.sigma;
  ppcg_status s = convert_csr_to_sell(n, nnz, d_rp, d_col, d_val, sigma, h->opts.precision != PPCG_FP64,
                                      h->opts.variant == PPCG_VARIANT_JACOBI_SCALED, stream, h->allocs, &h->sell,
                                      &h->A, &h->perm);
  // Matrix-free box stencil: a constant-coefficient box on a g^3 grid in grid row order,
  // solved by FP64 Alg. 2 on the grid path.
  bool box = false;
  if (s == PPCG_OK && want_box && h->opts.precision == PPCG_FP64 && h->opts.variant == PPCG_VARIANT_ALG2 &&
      !h->perm)
    box = detect_box_stencil(n, nnz, d_rp, d_col, d_val, stream, &h->box_g, &h->box_r, &h->box_cd, &h->box_co);
  free_tmp();
  if (s != PPCG_OK) { free_all(h); delete h; return s; }
  if (h->opts.format == PPCG_FMT_BOX &&
      (!box || h->opts.path == PPCG_PATH_CLUSTER || h->opts.path == PPCG_PATH_ONCHIP)) {
    free_all(h);
    delete h;
    set_error("ppcg_create: FMT_BOX needs a constant-coefficient box stencil in grid row order, FP64 Alg. 2 "
              "and the grid path");
    return PPCG_ERR_ARG;
  }

  // Execution plan (fixed for the handle, so every solve of it uses the same partition).
  // On chip: FP64 Alg. 2 whose vector tiles and matrix slots fit in one cluster's shared
  // memory; AUTO takes it whenever it fits (it removes every L2 round trip from an
  // iteration, the latency that bounds small systems).
  int path = h->opts.path;
  bool onchip_ok = false;
  if (h->opts.precision == PPCG_FP64 && h->opts.variant == PPCG_VARIANT_ALG2 &&
      (path == PPCG_PATH_AUTO || path == PPCG_PATH_ONCHIP)) {
    // 16 CTAs per cluster spread the FP64 work of an iteration over twice the SMs (the pass
    // is FP64-pipe bound on chip); it pays once every CTA has a few chunks.  8 otherwise, or
    // when the device cannot place a 16-CTA cluster with this much shared memory.
    const size_t limit = onchip_smem_limit(h->device);
    const size_t s8 = onchip_smem_bytes(h->A.nchunks, h->sell.onchip_slots, 8);
    const size_t s16 = onchip_smem_bytes(h->A.nchunks, h->sell.onchip_slots16, 16);
    const bool ok16 = s16 <= limit && h->sell.onchip_slots16 < INT32_MAX && onchip_cluster_fits(16, s16);
    const bool ok8 = s8 <= limit && h->sell.onchip_slots < INT32_MAX && onchip_cluster_fits(8, s8);
    if (ok16 && (h->A.nchunks >= 64 || !ok8)) { h->onchip_nc = 16; h->onchip_smem = s16; onchip_ok = true; }
    else if (ok8) { h->onchip_nc = 8; h->onchip_smem = s8; onchip_ok = true; }
  }
  if (path == PPCG_PATH_ONCHIP && !onchip_ok) {
    free_all(h);
    delete h;
    set_error("ppcg_create: PATH_ONCHIP needs FP64 Alg. 2 and a system that fits in one cluster's shared memory");
    return PPCG_ERR_ARG;
  }
  if (path == PPCG_PATH_AUTO && h->opts.format == PPCG_FMT_BOX) path = PPCG_PATH_GRID;
  if (path == PPCG_PATH_AUTO)
    path = onchip_ok ? PPCG_PATH_ONCHIP : n <= h->opts.cluster_max_rows ? PPCG_PATH_CLUSTER : PPCG_PATH_GRID;
  h->path = path;
  if (path != PPCG_PATH_GRID) box = false;
  if (!box) h->box_g = 0;
  if (path == PPCG_PATH_GRID) {
    // launch-shape tuning knob: an index among the plan's own kernels (SELL or box)
    const int nshapes = box ? grid_box_shape_count() : grid_shape_count();
    int k = 0;
    if (const char* e = getenv("PPCG_GRID_SHAPE")) k = atoi(e);
    if (k < 0 || k >= nshapes) k = 0;
    h->shape = box ? grid_box_shape_first() + k : k;
    // the offset pattern or the column dictionary, where the matrix has one, on the default
    // shape of the handle's precision; FP64 systems whose vector block exceeds half the L2
    // (so the row's own entries are not in L2 from the previous pass) get the pattern
    // kernel that prefetches them
    const bool streaming = (double)h->A.nchunks * kChunk * kSlots64 * sizeof(double) > 64.0 * 1024 * 1024;
    if (!box && k == 0)
      h->shape = grid_default_shape(h->A.pat_k > 0 ? PPCG_COLS_PATTERN : h->A.cidx ? PPCG_COLS_DICT : PPCG_COLS_SELL,
                                    h->opts.precision != PPCG_FP64, streaming);
    // One CTA per SM at most for small systems: enough warps for one 32-row chunk each,
    // so the grid barrier spans only the CTAs that have rows to work on.
    const int full = grid_blocks_for_device(h->device, h->shape);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    const int warps = grid_threads(h->shape) / 32;
    const int64_t need = (h->A.nchunks + warps - 1) / warps;
    h->grid = need >= sms ? full : (int)std::max<int64_t>(1, need);
    h->nparts = h->grid;
  } else {
    const int cc = h->opts.cluster_ctas;
    if (path == PPCG_PATH_CLUSTER && cc != 0 && cc != 2 && cc != 4 && cc != 8 && cc != 16) {
      free_all(h);
      delete h;
      set_error("ppcg_create: cluster_ctas must be 0 (tuned), 2, 4, 8 or 16");
      return PPCG_ERR_ARG;
    }
    h->cluster_cs = path == PPCG_PATH_CLUSTER && cc != 0 ? cc : kClusterSize;
    h->grid = h->cluster_cs;
    h->nparts = kClusterSize;
  }
  const bool fp32 = h->opts.precision != PPCG_FP64;
  const double v = fp32 ? 4.0 : 8.0;
  h->bytes_per_iter = (v + 4.0) * (double)nnz + 4.0 * (double)(n + 1) + 17.0 * v * (double)n;
  if (h->opts.variant == PPCG_VARIANT_JACOBI_SCALED)   // off-diagonals, 13 vector streams
    h->bytes_per_iter = (v + 4.0) * (double)(nnz - n) + 4.0 * (double)(n + 1) + 13.0 * v * (double)n;
  if (h->box_g > 0)   // no matrix: 17 vector streams + two stage arrays written and read
    h->bytes_per_iter = 21.0 * v * (double)n;

  // Workspace.
  SysDesc& d = h->desc;
  // Chunk-interleaved vector blocks.  FP64: r u wa wb z q s p x invd (also held by FP32_IR:
  // its outer residual, its solution, and the FP64 iteration it falls back to).  FP32_IR
  // adds the FP32 block r u wa wb z q s p d invd rhs.
  const bool scaled = h->opts.variant == PPCG_VARIANT_JACOBI_SCALED;
  h->ns64 = scaled ? kSlotsS : kSlots64;
  h->xslot = scaled ? kSlotXS : kSlotX64;
  const size_t rows_padded = (size_t)h->A.nchunks * kChunk;
  bool ok = walloc(h, &h->b_ws, n) && walloc(h, &h->tmp, n) &&
            walloc(h, &h->part, 2 * (size_t)h->nparts * 4) && walloc(h, &h->ctl, 1) &&
            walloc(h, &h->bar, 1) && walloc(h, &h->err, 1) && walloc(h, &h->d_desc, 1) &&
            walloc(h, &d.v64, rows_padded * h->ns64);
  if (ok && fp32) ok = walloc(h, &d.v32, rows_padded * kSlots32);
  if (ok && h->box_g > 0) ok = walloc(h, &d.box_t, 4 * (size_t)n);
  if (ok) {
    if (scaled)
      k_fill_scale_slots<<<blocks_for(n, 256), 256, 0, stream>>>(n, h->A.diag, d.v64, kSlotsS, kSlotDS, kSlotSigS);
    else
      k_to_slot<double><<<blocks_for(n, 256), 256, 0, stream>>>(n, nullptr, h->A.invd, d.v64, kSlots64, kSlotInvd);
    if (fp32)
      k_to_slot<float><<<blocks_for(n, 256), 256, 0, stream>>>(n, nullptr, h->A.invd32, d.v32, kSlots32, kSlotInvd);
    ok = cudaStreamSynchronize(stream) == cudaSuccess && cudaGetLastError() == cudaSuccess;
  }
  if (ok && !(h->stage = stage_get())) ok = false;
  if (!ok) {
    free_all(h);
    delete h;
    set_error("ppcg_create: out of device memory for the workspace");
    return PPCG_ERR_OOM;
  }
  d.A = h->A;
  d.precision = h->opts.precision;
  d.norm = h->opts.norm;
  // FP32 pipelined recurrences drift far faster than FP64 ones: unless the caller chose a
  // period, FP32_IR replaces residuals every 25 inner iterations and FP32_RU makes a
  // reliable update every 15 iterations.
  d.rr_period = h->opts.rr_period != 0                ? h->opts.rr_period
                : h->opts.precision == PPCG_FP32_IR ? 25
                : h->opts.precision == PPCG_FP32_RU ? 15
                                                    : 0;
  d.inner_maxit = h->opts.inner_maxit;
  d.max_outer = h->opts.max_outer;
  d.max_restarts = h->opts.max_restarts < 0 ? 0 : h->opts.max_restarts;
  d.variant = h->opts.variant;
  d.inner_tol = h->opts.inner_tol;
  d.gap_theta = h->opts.gap_theta == 0.0 ? 1e-6 : h->opts.gap_theta > 0.0 ? h->opts.gap_theta : 0.0;
  d.gap_fall = h->opts.gap_fall > 0 ? (double)h->opts.gap_fall : 100.0;
  d.onchip_slots = (int32_t)std::min<int64_t>(h->onchip_nc == 16 ? h->sell.onchip_slots16 : h->sell.onchip_slots,
                                               INT32_MAX);
  d.box_g = h->box_g;
  d.box_r = h->box_r;
  d.box_cd = h->box_cd;
  d.box_co = h->box_co;
  d.dmin = h->sell.dmin;
  d.dmax = h->sell.dmax;
  d.spin_limit_ns = h->opts.spin_limit_ns;
  d.nparts = h->nparts;
  d.part = h->part;
  d.ctl = h->ctl;
  d.bar = h->bar;
  d.err = h->err;
  if (path == PPCG_PATH_CLUSTER && h->opts.cluster_ctas == 0) {
    h->cluster_cs = tune_cluster_size(h, stream);
    h->grid = h->cluster_cs;
  }
  h->create_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_create).count();
  *handle = h;
  return PPCG_OK;
}

ppcg_status ppcg_plan_info(ppcg_handle h, ppcg_plan* out) {
  g_err[0] = 0;
  if (!h || !out) { set_error("ppcg_plan_info: NULL handle or plan"); return PPCG_ERR_ARG; }
  memset(out, 0, sizeof(*out));
  out->path = h->path;
  // the column source of the kernel that runs the iteration (a pattern matrix is also a
  // valid SELL matrix: the cluster and on-chip kernels read its stored columns)
  const bool grid = h->path == PPCG_PATH_GRID;
  out->columns = h->box_g > 0                                ? PPCG_COLS_MATRIX_FREE
                 : grid                                     ? grid_shape_cols(h->shape)
                                                            : PPCG_COLS_SELL;
  out->sigma = h->sell.sigma;
  out->pattern_k = h->A.pat_k;
  out->dict_size = h->sell.col_dict;
  out->ctas = h->path == PPCG_PATH_GRID ? h->grid : (h->path == PPCG_PATH_ONCHIP ? h->onchip_nc : h->cluster_cs);
  out->slots = h->sell.nslots;
  out->padding = h->sell.padding;
  out->convert_seconds = h->sell.seconds;
  out->create_seconds = h->create_seconds;
  out->bytes_per_iter = h->bytes_per_iter;
  return PPCG_OK;
}

ppcg_status ppcg_solve(ppcg_handle h, const double* b, const double* x0, double* x, double tol,
                       int32_t maxit, cudaStream_t st, ppcg_info* info) {
  NvtxRange nvtx_range("ppcg_solve");
  g_err[0] = 0;
  if (!h) { set_error("ppcg_solve: NULL handle"); return PPCG_ERR_ARG; }
  if (!(tol >= 0.0) || maxit < 0 || (h->n > 0 && (!b || !x))) {
    set_error("ppcg_solve: bad arguments (tol=%g maxit=%d)", tol, maxit);
    return PPCG_ERR_ARG;
  }
  if (h->n == 0) { write_trivial_info(info, PPCG_OK); h->last_solve = 2; return PPCG_OK; }
  h->stream = st;
  ppcg_status s = stage_inputs(h, b, x0, false, st);
  if (s != PPCG_OK) return s;
  prepare_control(h, tol, maxit, st);
  cudaMemcpyAsync(h->d_desc, &h->desc, sizeof(SysDesc), cudaMemcpyHostToDevice, st);
  cudaError_t e;
  if (h->path == PPCG_PATH_GRID) {
    e = launch_grid(h->d_desc, h->shape, h->grid, 0, st);
  } else if (h->path == PPCG_PATH_ONCHIP) {
    const int32_t* d_list = single_work_list();
    if (!d_list) { set_error("ppcg_solve: could not allocate the cluster work list"); return PPCG_ERR_OOM; }
    e = launch_onchip(h->d_desc, d_list, d_list + 1, 1, 0, h->onchip_smem, h->onchip_nc, st);
  } else {
    const int32_t* d_list = single_work_list();
    if (!d_list) { set_error("ppcg_solve: could not allocate the cluster work list"); return PPCG_ERR_OOM; }
    e = launch_clusters(h->d_desc, d_list, d_list + 1, 1, 0, st, /*spread=*/true, nullptr, 0, h->cluster_cs);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("ppcg_solve: launch failed: %s", cudaGetErrorString(e));
    return PPCG_ERR_CUDA;
  }
  stage_outputs(h, x, st);
  if (info) {
    std::vector<std::pair<ppcg_ctx*, ppcg_info*>> items{{h, info}};
    enqueue_info(items, st);
  } else {
    enqueue_stage_copies(h, st);
  }
  return check_launch("ppcg_solve") ? PPCG_OK : PPCG_ERR_CUDA;
}

ppcg_status ppcg_last_info(ppcg_handle h, ppcg_info* info) {
  g_err[0] = 0;
  if (!h || !info) { set_error("ppcg_last_info: NULL handle or info"); return PPCG_ERR_ARG; }
  if (h->last_solve == 2) { write_trivial_info(info, PPCG_OK); return PPCG_OK; }
  if (h->last_solve != 1 || !h->stage) { set_error("ppcg_last_info: the handle has not solved yet"); return PPCG_ERR_ARG; }
  const InfoJob j{h->stage, info, h->bytes_per_iter, h->opts.norm, h->opts.precision};
  fill_info(*h->stage, j, info);
  return PPCG_OK;
}

ppcg_status ppcg_batch_solve(int32_t count, const ppcg_handle* hs, const double* const* b,
                             const double* const* x0, double* const* x, const double* tol,
                             const int32_t* maxit, cudaStream_t st, ppcg_info* infos) {
  NvtxRange nvtx_range("ppcg_batch_solve");
  g_err[0] = 0;
  if (count < 0 || (count > 0 && (!hs || !b || !x || !tol || !maxit))) {
    set_error("ppcg_batch_solve: bad arguments");
    return PPCG_ERR_ARG;
  }
  for (int i = 0; i < count; i++) {
    if (!hs[i] || !(tol[i] >= 0.0) || maxit[i] < 0 || (hs[i]->n > 0 && (!b[i] || !x[i]))) {
      set_error("ppcg_batch_solve: bad arguments for system %d", i);
      return PPCG_ERR_ARG;
    }
    for (int j = 0; j < i; j++)
      if (hs[j] == hs[i]) { set_error("ppcg_batch_solve: handle %d repeated", i); return PPCG_ERR_ARG; }
  }
  std::vector<int> cl, gr, oc;
  for (int i = 0; i < count; i++) {
    ppcg_ctx* h = hs[i];
    if (h->n == 0) { if (infos) write_trivial_info(&infos[i], PPCG_OK); continue; }
    if (!is_device_ptr(x[i])) { set_error("ppcg_batch_solve: x[%d] must be a device pointer", i); return PPCG_ERR_ARG; }
    h->stream = st;
    ppcg_status s = stage_inputs(h, b[i], x0 ? x0[i] : nullptr, true, st);
    if (s != PPCG_OK) return s;
    prepare_control(h, tol[i], maxit[i], st);
    (h->path == PPCG_PATH_CLUSTER ? cl : h->path == PPCG_PATH_ONCHIP ? oc : gr).push_back(i);
  }
  // On-chip systems: one launch of clusters per cluster size (one system per cluster at a
  // time, longest first) on a side stream, overlapping the cluster-path launch below.
  cudaEvent_t oc_done = nullptr;
  if (!oc.empty()) {
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr;
    if (!side_stream(hs[oc[0]]->device, &side, &fork, &oc_done)) {
      set_error("ppcg_batch_solve: could not create the side stream");
      return PPCG_ERR_CUDA;
    }
    cudaEventRecord(fork, st);
    cudaStreamWaitEvent(side, fork, 0);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, hs[oc[0]]->device);
    cudaError_t e = cudaSuccess;
    for (int nc : {16, 8}) {
      std::vector<int> grp;
      for (int i : oc)
        if (hs[i]->onchip_nc == nc) grp.push_back(i);
      if (grp.empty() || e != cudaSuccess) continue;
      const int m = (int)grp.size();
      std::vector<SysDesc> descs(m);
      size_t smem = 0;
      std::vector<int> order(m);
      for (int k = 0; k < m; k++) {
        descs[k] = hs[grp[k]]->desc;
        smem = std::max(smem, hs[grp[k]]->onchip_smem);
        order[k] = k;
      }
      const int nclusters = std::max(1, std::min(m, sms / nc));
      std::stable_sort(order.begin(), order.end(),
                       [&](int a, int c) { return hs[grp[a]]->sell.nslots > hs[grp[c]]->sell.nslots; });
      std::vector<std::vector<int>> lists(nclusters);
      std::vector<double> load(nclusters, 0.0);
      for (int k : order) {
        const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lists[c].push_back(k);
        load[c] += (double)hs[grp[k]]->sell.nslots + 32.0 * (double)hs[grp[k]]->n;
      }
      std::vector<int32_t> flat, ptr(1, 0);
      for (auto& l : lists) { for (int k : l) flat.push_back(k); ptr.push_back((int32_t)flat.size()); }
      std::vector<int32_t> packed(ptr);
      packed.insert(packed.end(), flat.begin(), flat.end());
      SysDesc* d_descs = nullptr;
      int32_t* d_lists = nullptr;
      if (cudaMallocAsync((void**)&d_descs, m * sizeof(SysDesc), side) != cudaSuccess ||
          cudaMallocAsync((void**)&d_lists, packed.size() * sizeof(int32_t), side) != cudaSuccess) {
        cudaGetLastError();
        cudaEventRecord(oc_done, side);
        cudaStreamWaitEvent(st, oc_done, 0);
        set_error("ppcg_batch_solve: out of device memory for the schedule");
        return PPCG_ERR_OOM;
      }
      cudaMemcpyAsync(d_descs, descs.data(), m * sizeof(SysDesc), cudaMemcpyHostToDevice, side);
      cudaMemcpyAsync(d_lists, packed.data(), packed.size() * sizeof(int32_t), cudaMemcpyHostToDevice, side);
      e = launch_onchip(d_descs, d_lists + ptr.size(), d_lists, nclusters, 0, smem, nc, side);
      cudaFreeAsync(d_descs, side);
      cudaFreeAsync(d_lists, side);
    }
    cudaEventRecord(oc_done, side);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaStreamWaitEvent(st, oc_done, 0);
      set_error("ppcg_batch_solve: on-chip launch failed: %s", cudaGetErrorString(e));
      return PPCG_ERR_CUDA;
    }
  }
  // Cluster-path systems: one persistent launch per cluster size in the batch (the sizes
  // the handles' plans fixed), largest size first, each on its own stream: the launch of
  // the largest clusters (the largest systems) fills the GPU first and the next ones take
  // the SMs its clusters give up as its work list drains.  Within a launch, systems are
  // ordered longest first by an estimate.  Up to two systems per cluster: a static
  // longest-processing-time assignment (each cluster's first system is one of the longest,
  // the rest fill the least loaded clusters), which leaves the critical longest solves the
  // least contended.  More: the clusters take systems from a shared counter (list
  // scheduling, which absorbs the estimate's errors; 1,024 systems: 1.78 -> 1.19 s).
  // Results depend on neither.
  std::vector<cudaEvent_t> joins;
  if (!cl.empty()) {
    std::vector<int> sizes;
    for (int i : cl)
      if (std::find(sizes.begin(), sizes.end(), hs[i]->cluster_cs) == sizes.end()) sizes.push_back(hs[i]->cluster_cs);
    std::sort(sizes.rbegin(), sizes.rend());
    for (size_t gi = 0; gi < sizes.size(); gi++) {
      const int cs = sizes[gi];
      std::vector<int> grp;
      for (int i : cl)
        if (hs[i]->cluster_cs == cs) grp.push_back(i);
      cudaStream_t gs = st;
      if (gi > 0) {
        cudaEvent_t fork = nullptr, join = nullptr;
        if (!side_stream(hs[grp[0]]->device, &gs, &fork, &join, (int)gi)) {
          for (cudaEvent_t j : joins) cudaStreamWaitEvent(st, j, 0);
          set_error("ppcg_batch_solve: could not create a side stream");
          return PPCG_ERR_CUDA;
        }
        cudaEventRecord(fork, st);
        cudaStreamWaitEvent(gs, fork, 0);
        joins.push_back(join);
      }
      const int m = (int)grp.size();
      std::vector<SysDesc> descs(m);
      std::vector<double> cost(m);
      for (int k = 0; k < m; k++) {
        descs[k] = hs[grp[k]]->desc;
        cost[k] = cluster_solve_cost(hs[grp[k]], 0);
      }
      const int nclusters = std::max(1, std::min(m, max_active_clusters(hs[grp[0]]->device, cs)));
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
      SysDesc* d_descs = nullptr;
      int32_t* d_lists = nullptr;
      cudaError_t e = cudaSuccess;
      if (cudaMallocAsync((void**)&d_descs, m * sizeof(SysDesc), gs) != cudaSuccess ||
          cudaMallocAsync((void**)&d_lists, packed.size() * sizeof(int32_t), gs) != cudaSuccess) {
        cudaGetLastError();
        e = cudaErrorMemoryAllocation;
      } else {
        cudaMemcpyAsync(d_descs, descs.data(), m * sizeof(SysDesc), cudaMemcpyHostToDevice, gs);
        cudaMemcpyAsync(d_lists, packed.data(), packed.size() * sizeof(int32_t), cudaMemcpyHostToDevice, gs);
        e = dynamic ? launch_clusters(d_descs, d_lists, nullptr, nclusters, 0, gs, false, d_lists + m, m, cs)
                    : launch_clusters(d_descs, d_lists + nclusters + 1, d_lists, nclusters, 0, gs, false, nullptr, 0,
                                      cs);
        cudaFreeAsync(d_descs, gs);
        cudaFreeAsync(d_lists, gs);
      }
      if (gi > 0) cudaEventRecord(joins.back(), gs);
      if (e != cudaSuccess) {
        cudaGetLastError();
        for (cudaEvent_t j : joins) cudaStreamWaitEvent(st, j, 0);
        if (oc_done) cudaStreamWaitEvent(st, oc_done, 0);
        set_error(e == cudaErrorMemoryAllocation ? "ppcg_batch_solve: out of device memory for the schedule"
                                                 : "ppcg_batch_solve: cluster launch failed: %s",
                  cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? PPCG_ERR_OOM : PPCG_ERR_CUDA;
      }
    }
  }
  // Grid-path systems: one whole-GPU launch each.
  for (int i : gr) {
    ppcg_ctx* h = hs[i];
    cudaMemcpyAsync(h->d_desc, &h->desc, sizeof(SysDesc), cudaMemcpyHostToDevice, st);
    cudaError_t e = launch_grid(h->d_desc, h->shape, h->grid, 0, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("ppcg_batch_solve: launch failed: %s", cudaGetErrorString(e));
      return PPCG_ERR_CUDA;
    }
  }
  if (oc_done) cudaStreamWaitEvent(st, oc_done, 0);
  for (cudaEvent_t j : joins) cudaStreamWaitEvent(st, j, 0);
  std::vector<std::pair<ppcg_ctx*, ppcg_info*>> items;
  for (int i = 0; i < count; i++) {
    if (hs[i]->n == 0) { hs[i]->last_solve = 2; continue; }
    stage_outputs(hs[i], x[i], st);
    items.push_back({hs[i], infos ? &infos[i] : nullptr});
  }
  if (!items.empty()) enqueue_info(items, st);
  return check_launch("ppcg_batch_solve") ? PPCG_OK : PPCG_ERR_CUDA;
}

ppcg_status ppcg_selftest_barrier_timeout(int32_t grid, int32_t drop_rank, int64_t limit_ns,
                                          int32_t* timed_out) {
  g_err[0] = 0;
  if (grid < 2 || grid > 4096 || drop_rank < 0 || drop_rank >= grid || limit_ns <= 0 || !timed_out) {
    set_error("ppcg_selftest_barrier_timeout: bad arguments");
    return PPCG_ERR_ARG;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (grid > sms) grid = sms;   // one CTA per SM keeps the cooperative launch valid
  if (drop_rank >= grid) drop_rank = grid - 1;
  unsigned* bar = nullptr;
  int32_t* err = nullptr;
  int32_t* out = nullptr;
  if (cudaMalloc(&bar, sizeof(unsigned)) != cudaSuccess || cudaMalloc(&err, sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&out, grid * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(bar); cudaFree(err); cudaFree(out);
    set_error("ppcg_selftest_barrier_timeout: out of device memory");
    return PPCG_ERR_OOM;
  }
  cudaMemset(bar, 0, sizeof(unsigned));
  cudaMemset(err, 0, sizeof(int32_t));
  cudaMemset(out, 0xff, grid * sizeof(int32_t));
  cudaError_t e = launch_barrier_selftest(bar, err, out, grid, drop_rank, limit_ns, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  std::vector<int32_t> h(grid);
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), out, grid * sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaFree(bar); cudaFree(err); cudaFree(out);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("ppcg_selftest_barrier_timeout: %s", cudaGetErrorString(e));
    return PPCG_ERR_CUDA;
  }
  int32_t n = 0;
  for (int i = 0; i < grid; i++) n += (i != drop_rank && h[i] == 0);
  *timed_out = n;
  return PPCG_OK;
}

void ppcg_destroy(ppcg_handle h) {
  if (!h) return;
  // the handle's work is ordered on its last stream: wait for that stream only
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) cudaGetLastError();
  free_all(h);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) cudaGetLastError();
  delete h;
}

}  // extern "C"
