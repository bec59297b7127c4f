// Solver handle internals shared by the ABI layer (api.cu) and the server (server.cu).
#pragma once
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "internal.h"

namespace ppcg {

// Host-side copy of the device control block + launch error flag (pinned).
struct Stage {
  Ctl ctl;
  int32_t err;
  int32_t pad;
};

struct InfoJob {
  Stage* stage;
  ppcg_info* info;
  double bytes_per_iter;
  int32_t norm;
  int32_t precision;
};

inline void fill_info(const Stage& s, const InfoJob& j, ppcg_info* out) {
  ppcg_info r;
  memset(&r, 0, sizeof(r));
  const Ctl& c = s.ctl;
  r.status = s.err != 0 ? s.err : c.status;
  r.iters = c.iter;
  r.outer_iters = c.outer;
  r.rr_count = c.rr_count;
  r.bnorm = c.bnorm;
  if (j.precision == PPCG_FP32_IR) {
    r.rel_res_recursive = c.bnorm > 0 ? c.rn / c.bnorm : 0.0;
  } else {
    r.rel_res_recursive = j.norm == PPCG_NORM_PAPER_U_ABS ? c.norm : (c.bnorm > 0 ? c.norm / c.bnorm : 0.0);
  }
  r.rel_res_true = c.bnorm > 0 ? c.res_true / c.bnorm : 0.0;
  r.seconds = c.t_end > c.t_start ? (double)(c.t_end - c.t_start) * 1e-9 : 0.0;
  r.bytes_per_iter = j.bytes_per_iter;
  r.fp64_fallback = c.fallback;
  *out = r;
}

}  // namespace ppcg

struct ppcg_ctx {
  int device = 0;
  int64_t n = 0, nnz = 0;
  ppcg_opts opts;
  ppcg::SellBuild sell;
  ppcg::DevMatrix A;
  int32_t* perm = nullptr;
  std::vector<void*> allocs;
  int32_t path = PPCG_PATH_GRID;
  size_t onchip_smem = 0;   // dynamic shared memory per CTA of the on-chip path
  int onchip_nc = 8;        // CTAs per on-chip cluster (8 or 16)
  int cluster_cs = 8;       // CTAs per cluster of the CLUSTER path (2, 4, 8 or 16)
  int64_t tune_key = 0;     // cluster-size cache key (0: not tuned)
  int32_t box_g = 0, box_r = 0;      // matrix-free box stencil (box_g > 0)
  double box_cd = 0.0, box_co = 0.0;
  int shape = 0;       // grid-path launch shape (index into the kernel variants)
  int grid = 0;        // CTAs of the grid path
  int nparts = 0;      // partial slots per pass (CTAs in the group)
  double bytes_per_iter = 0.0;
  // workspace
  double *b_ws = nullptr, *tmp = nullptr;
  int ns64 = 0, xslot = 0;   // slots of the FP64 vector block and the slot holding x
  double* part = nullptr;
  ppcg::Ctl* ctl = nullptr;
  unsigned* bar = nullptr;
  int32_t* err = nullptr;
  ppcg::SysDesc* d_desc = nullptr;
  ppcg::SysDesc desc;        // host copy, refreshed per solve
  ppcg::Stage* stage = nullptr;   // pinned, from the library's stage pool
  cudaStream_t stream = nullptr;  // stream of the handle's latest work (creation or solve)
  int32_t last_solve = 0;   // ppcg_last_info source: 0 none, 1 the stage, 2 a trivial OK (n = 0)
  double create_seconds = 0.0;   // wall time of ppcg_create (ppcg_plan_info)
};


namespace ppcg {

// Enqueue b/x0 into solver-order device storage (fills h->desc.b and x_zero; x0 goes into
// the x slot of the vector block).  require_device: b and x0 must be device pointers.
ppcg_status stage_inputs(ppcg_ctx* h, const double* b, const double* x0, bool require_device, cudaStream_t st);
// Enqueue the copy (and un-permutation) of the solver's x into the caller's x (host or device).
void stage_outputs(ppcg_ctx* h, double* x, cudaStream_t st);
// Enqueue a fresh control block and the barrier/err reset for a new solve.
void prepare_control(ppcg_ctx* h, double tol, int32_t maxit, cudaStream_t st);
// Device bytes a handle of this size will allocate (estimate used for admission).
size_t footprint_bytes(int64_t n, int64_t nnz, int32_t precision);
bool is_device_ptr(const void* p);

// Estimated device time of a cluster-path solve (iterations = 0: the whole solve), used only
// to order the clusters' work queue.  Iterations grow like the grid side, n^(1/2) for 2-D
// stencils (about 4 off-diagonals per row) and n^(1/3) for 3-D ones and geometric graphs;
// an iteration costs a fixed ~8 us of control and barriers plus its bytes at ~100 GB/s (a
// cluster's share of HBM when the GPU is full).
inline double cluster_solve_cost(const ppcg_ctx* h, double iterations) {
  const double n = (double)(h->n > 0 ? h->n : 1);
  const double offdiag = (double)(h->nnz - h->n) / n;
  const double it = iterations > 0 ? iterations : 4.3 * std::pow(n, offdiag <= 4.5 ? 0.5 : 1.0 / 3.0);
  const double v = h->opts.precision == PPCG_FP64 ? 8.0 : 4.0;
  const double bytes = (double)h->sell.nslots * (v + 4.0) + 17.0 * v * n;
  return it * (8e-6 + bytes / 1e11);
}

}  // namespace ppcg
