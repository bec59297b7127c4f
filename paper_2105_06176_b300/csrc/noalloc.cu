// Allocation-free solve entry point (ppcg_solve_noalloc in include/ppcg.h).
//
// Some callers cannot allocate device memory at solve time: code running under a
// framework that owns every device allocation through its own pool, real-time loops that
// forbid cudaMalloc/cudaFree (both may synchronise the whole device), or plug-ins whose
// host rules out allocation after initialisation.  For them this file offers a pipelined
// PCG solve (Algorithm 2 of arXiv 2105.06176, Jacobi preconditioner) that works straight
// from the caller's device CSR and keeps all of its working vectors in one statically
// sized device array declared below.  It never calls cudaMalloc, cudaFree or an allocating
// library routine.
//
// The scratch array exists once per GPU that loads this library and stays allocated until
// the process exits.  All calls on a device share it: two calls whose work overlaps on the
// GPU (different streams, or different host threads) race on it and corrupt each other's
// results, so callers must order them.  Every call rewrites whatever it reads before
// reading it, so leftovers of an earlier call never leak into a result.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace {

constexpr int64_t kNoAllocMaxRows = 1 << 16;       // 65,536 rows
constexpr int kNaCluster = 8;                      // CTAs in the single cluster
constexpr int kNaThreads = 256;
constexpr int kNaVectors = 9;                      // r u wa wb z q s p invd
// Layout of the scratch array (in doubles): 9 vectors of kNoAllocMaxRows, then two
// buffers of per-CTA partial sums, then the result record.
constexpr int64_t kPartOff = kNaVectors * kNoAllocMaxRows;
constexpr int64_t kResultOff = kPartOff + 2 * kNaCluster * 4;
constexpr int64_t kScratchDoubles = kResultOff + 16;
constexpr int kBadArg = 1, kBadDiag = 2;           // validation flags of the first phase

// 4.5 MiB per device.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

struct NaResult {        // overlays g_noalloc_scratch[kResultOff ...]
  double status, iters, bnorm, res_rec, res_true, t_ns;
};

__device__ __forceinline__ unsigned long long na_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void na_cluster_sync() {
  __syncthreads();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned na_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Block sum of three values (fixed tree), written by thread 0 to slot[0..2].
__device__ void na_block_partials(double a0, double a1, double a2, double* slot, double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_down_sync(0xffffffffu, a0, o);
    a1 += __shfl_down_sync(0xffffffffu, a1, o);
    a2 += __shfl_down_sync(0xffffffffu, a2, o);
  }
  if (lane == 0) { sm[warp * 3] = a0; sm[warp * 3 + 1] = a1; sm[warp * 3 + 2] = a2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < nw; w++) { s0 += sm[w * 3]; s1 += sm[w * 3 + 1]; s2 += sm[w * 3 + 2]; }
    slot[0] = s0; slot[1] = s1; slot[2] = s2;
  }
}

// Sum of the cluster's partial slots in rank order; identical bits in every CTA.
__device__ void na_reduce(const double* part, double out[3]) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int k = 0; k < kNaCluster; k++) {
    s0 += __ldcg(part + 4 * k);
    s1 += __ldcg(part + 4 * k + 1);
    s2 += __ldcg(part + 4 * k + 2);
  }
  out[0] = s0; out[1] = s1; out[2] = s2;
}

// (A v)_i over the caller's CSR row, terms in CSR order; gathers through L2 (other CTAs
// wrote v in the previous phase).
__device__ __forceinline__ double na_row(const int64_t* rp, const int32_t* col, const double* val,
                                         const double* v, int64_t i) {
  double acc = 0.0;
  for (int64_t k = rp[i]; k < rp[i + 1]; k++) acc = fma(val[k], __ldcg(v + col[k]), acc);
  return acc;
}

// One cluster of 8 CTAs runs the whole solve: the setup of Alg. 2, then one fused phase per
// iteration (vector updates, dot products, preconditioner and SpMV) with alpha/beta formed in
// every CTA from the same partials, a cluster barrier between phases, and the final true
// residual.
__global__ void __cluster_dims__(kNaCluster, 1, 1) __launch_bounds__(kNaThreads)
k_solve_noalloc(int64_t n, int64_t nnz, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                const double* __restrict__ val, const double* __restrict__ b, const double* x0,
                double* x, double tol, int32_t maxit) {
  __shared__ double sm[3 * 32];
  __shared__ int bad;
  double* S = g_noalloc_scratch;
  double* r = S;
  double* u = S + kNoAllocMaxRows;
  double* wv[2] = {S + 2 * kNoAllocMaxRows, S + 3 * kNoAllocMaxRows};
  double* z = S + 4 * kNoAllocMaxRows;
  double* q = S + 5 * kNoAllocMaxRows;
  double* s = S + 6 * kNoAllocMaxRows;
  double* p = S + 7 * kNoAllocMaxRows;
  double* invd = S + 8 * kNoAllocMaxRows;
  double* part = S + kPartOff;
  NaResult* res = reinterpret_cast<NaResult*>(S + kResultOff);
  const unsigned rank = na_rank();
  const int64_t t0 = (int64_t)rank * blockDim.x + threadIdx.x;
  const int64_t T = (int64_t)kNaCluster * blockDim.x;
  const unsigned long long start = na_timer();
  int parity = 0;
  double red[3];
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();

  // Validation of the caller's CSR, the Jacobi diagonal and x0 (x may alias x0).  A row's
  // columns are read only once its pointers are known to lie in [0, nnz], and no phase
  // below gathers anything unless every row passed: a malformed matrix ends the call with
  // PPCG_ERR_ARG before any vector is indexed by a column, and a missing or non-positive
  // diagonal entry with PPCG_ERR_NOT_SPD.
  for (int64_t i = t0; i < n; i += T) {
    const int64_t a = rp[i], e = rp[i + 1];
    int f = 0;
    if (a < 0 || e < a || e > nnz || (i == 0 && a != 0) || (i == n - 1 && e != nnz)) f |= kBadArg;
    double d = 0.0;
    bool found = false;
    if (!(f & kBadArg)) {
      for (int64_t k = a; k < e; k++) {
        const int32_t c = col[k];
        if (c < 0 || c >= n) f |= kBadArg;
        else if (c == i) { d += val[k]; found = true; }
      }
    }
    if (!found || !(d > 0.0)) f |= kBadDiag;
    invd[i] = f == 0 ? 1.0 / d : 0.0;
    x[i] = x0 ? x0[i] : 0.0;
    if (f) atomicOr(&bad, f);
  }
  na_cluster_sync();
  // Every CTA must agree on the checks: share the flags through the partials.
  {
    double* slot = part + (parity * kNaCluster + rank) * 4;
    if (threadIdx.x == 0) {
      slot[0] = (bad & kBadArg) ? 1.0 : 0.0;
      slot[1] = (bad & kBadDiag) ? 1.0 : 0.0;
      slot[2] = 0.0;
    }
    na_cluster_sync();
    na_reduce(part + parity * kNaCluster * 4, red);
    parity ^= 1;
  }
  int status = PPCG_ERR_NOT_CONVERGED;
  int it = 0;
  double bnorm = 0.0, gamma = 0.0, delta = 0.0, norm = 0.0, gamma_prev = 0.0, alpha_prev = 0.0;
  bool done = false;
  if (red[0] != 0.0) { status = PPCG_ERR_ARG; done = true; }
  else if (red[1] != 0.0) { status = PPCG_ERR_NOT_SPD; done = true; }

  if (!done) {
    // setup, first half: r0 = b - A x0; u0 = M^-1 r0; partial (b, b)
    double pb = 0.0;
    for (int64_t i = t0; i < n; i += T) {
      double ri = b[i] - na_row(rp, col, val, x, i);
      r[i] = ri;
      u[i] = invd[i] * ri;
      pb = fma(b[i], b[i], pb);
    }
    na_block_partials(pb, 0.0, 0.0, part + (parity * kNaCluster + rank) * 4, sm);
    na_cluster_sync();
    na_reduce(part + parity * kNaCluster * 4, red);
    parity ^= 1;
    bnorm = sqrt(red[0]);
    if (bnorm == 0.0) {            // A x = 0 has the solution x = 0
      for (int64_t i = t0; i < n; i += T) x[i] = 0.0;
      status = PPCG_OK;
      done = true;
      na_cluster_sync();           // the final residual below gathers x
    }
  }
  if (!done) {
    // setup: w0 = A u0; gamma0 = (r0, u0); delta = (w0, u0); ||r0||
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t i = t0; i < n; i += T) {
      double wi = na_row(rp, col, val, u, i);
      wv[0][i] = wi;
      a0 = fma(r[i], u[i], a0);
      a1 = fma(wi, u[i], a1);
      a2 = fma(r[i], r[i], a2);
    }
    na_block_partials(a0, a1, a2, part + (parity * kNaCluster + rank) * 4, sm);
    na_cluster_sync();
    na_reduce(part + parity * kNaCluster * 4, red);
    parity ^= 1;
    gamma = red[0]; delta = red[1]; norm = sqrt(red[2]);
  }
  while (!done) {
    if (norm <= tol * bnorm) { status = PPCG_OK; break; }
    if (it >= maxit) { status = PPCG_ERR_NOT_CONVERGED; break; }
    if (!isfinite(gamma) || !isfinite(delta)) { status = PPCG_ERR_NONFINITE; break; }
    double alpha, beta;
    if (it > 0) {
      beta = gamma / gamma_prev;
      double den = delta - beta * gamma / alpha_prev;
      if (!(gamma > 0.0) || !(den > 0.0)) { status = PPCG_ERR_BREAKDOWN; break; }
      alpha = gamma / den;
    } else {
      beta = 0.0;
      if (!(gamma > 0.0) || !(delta > 0.0)) { status = PPCG_ERR_BREAKDOWN; break; }
      alpha = gamma / delta;
    }
    const double* wc = wv[it & 1];
    double* wn = wv[(it + 1) & 1];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t i = t0; i < n; i += T) {
      // preconditioner and SpMV of the previous step, fused: n_i = (A M^-1 w)_i
      double ni = 0.0;
      for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
        int32_t c = col[k];
        ni = fma(val[k], __ldcg(invd + c) * __ldcg(wc + c), ni);
      }
      const double wi = __ldcg(wc + i);
      const double mi = invd[i] * wi;
      const double zi = it > 0 ? fma(beta, z[i], ni) : ni;
      const double qi = it > 0 ? fma(beta, q[i], mi) : mi;
      const double si = it > 0 ? fma(beta, s[i], wi) : wi;
      const double pi = it > 0 ? fma(beta, p[i], u[i]) : u[i];
      x[i] = fma(alpha, pi, x[i]);
      const double ri = fma(-alpha, si, r[i]);
      const double ui = fma(-alpha, qi, u[i]);
      const double wni = fma(-alpha, zi, wi);
      z[i] = zi; q[i] = qi; s[i] = si; p[i] = pi;
      r[i] = ri; u[i] = ui; wn[i] = wni;
      a0 = fma(ri, ui, a0);
      a1 = fma(wni, ui, a1);
      a2 = fma(ri, ri, a2);
    }
    na_block_partials(a0, a1, a2, part + (parity * kNaCluster + rank) * 4, sm);
    na_cluster_sync();
    na_reduce(part + parity * kNaCluster * 4, red);
    parity ^= 1;
    gamma_prev = gamma;
    alpha_prev = alpha;
    gamma = red[0]; delta = red[1]; norm = sqrt(red[2]);
    it++;
  }
  // final true residual ||b - A x||
  double res_true = 0.0;
  if (status != PPCG_ERR_NOT_SPD && status != PPCG_ERR_ARG) {
    double a0 = 0.0;
    for (int64_t i = t0; i < n; i += T) {
      double t = b[i] - na_row(rp, col, val, x, i);
      a0 = fma(t, t, a0);
    }
    na_block_partials(a0, 0.0, 0.0, part + (parity * kNaCluster + rank) * 4, sm);
    na_cluster_sync();
    na_reduce(part + parity * kNaCluster * 4, red);
    res_true = sqrt(red[0]);
  }
  if (rank == 0 && threadIdx.x == 0) {
    res->status = (double)status;
    res->iters = (double)it;
    res->bnorm = bnorm;
    res->res_rec = norm;
    res->res_true = res_true;
    res->t_ns = (double)(na_timer() - start);
  }
  na_cluster_sync();   // no CTA leaves while others may still read the partials
}

std::mutex g_setup_mu;
void* g_scratch_addr[64] = {nullptr};

// Once per device, with that device current: look up the scratch array's device address
// and make the driver load this file's kernel.  With lazy module loading (the CUDA
// default) the module -- the scratch array among its globals -- is brought onto the
// device by the first use of one of its symbols, which allocates; doing both lookups here
// keeps every later call free of that work.
ppcg_status noalloc_setup(void** scratch) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    ppcg::set_error("ppcg_solve_noalloc: no current CUDA device");
    return PPCG_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* addr = nullptr;
    e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e == cudaSuccess) {
      cudaFuncAttributes fa;
      e = cudaFuncGetAttributes(&fa, k_solve_noalloc);
    }
    if (e != cudaSuccess) {
      ppcg::set_error("ppcg_solve_noalloc: device set-up failed: %s", cudaGetErrorString(e));
      return PPCG_ERR_CUDA;
    }
    g_scratch_addr[dev] = addr;
  }
  *scratch = g_scratch_addr[dev];
  return PPCG_OK;
}

}  // namespace

extern "C" ppcg_status ppcg_solve_noalloc(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col,
                                          const double* val, const double* b, const double* x0, double* x,
                                          double tol, int32_t maxit, cudaStream_t stream, ppcg_info* info) {
  using ppcg::set_error;
  if (n > kNoAllocMaxRows) {
    set_error("ppcg_solve_noalloc: n = %lld exceeds the allocation-free limit of %lld rows; use ppcg_create/ppcg_solve",
              (long long)n, (long long)kNoAllocMaxRows);
    return PPCG_ERR_ARG;
  }
  if (n < 0 || nnz < 0 || !(tol >= 0.0) || maxit < 0 || (n > 0 && (!row_ptr || !col || !val || !b || !x))) {
    set_error("ppcg_solve_noalloc: bad arguments");
    return PPCG_ERR_ARG;
  }
  void* scratch = nullptr;
  const ppcg_status st = noalloc_setup(&scratch);   // also on n = 0: the set-up call
  if (st != PPCG_OK) return st;
  if (n == 0) {
    if (info) { memset(info, 0, sizeof(*info)); info->status = PPCG_OK; }
    return PPCG_OK;
  }
  k_solve_noalloc<<<kNaCluster, kNaThreads, 0, stream>>>(n, nnz, row_ptr, col, val, b, x0, x, tol, maxit);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("ppcg_solve_noalloc: launch failed: %s", cudaGetErrorString(e));
    return PPCG_ERR_CUDA;
  }
  if (info) {
    NaResult r;
    e = cudaMemcpyAsync(&r, static_cast<double*>(scratch) + kResultOff, sizeof(r), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
      set_error("ppcg_solve_noalloc: %s", cudaGetErrorString(e));
      return PPCG_ERR_CUDA;
    }
    memset(info, 0, sizeof(*info));
    info->status = (int32_t)r.status;
    info->iters = (int32_t)r.iters;
    info->bnorm = r.bnorm;
    info->rel_res_recursive = r.bnorm > 0 ? r.res_rec / r.bnorm : 0.0;
    info->rel_res_true = r.bnorm > 0 ? r.res_true / r.bnorm : 0.0;
    info->seconds = r.t_ns * 1e-9;
    info->bytes_per_iter = 12.0 * (double)nnz + 4.0 * (double)(n + 1) + 17.0 * 8.0 * (double)n;
  }
  return PPCG_OK;
}
