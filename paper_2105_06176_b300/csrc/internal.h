// Internal declarations shared by the library's translation units (not installed).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/ppcg.h"

namespace ppcg {

constexpr int kChunk = 32;           // SELL-C-sigma chunk height C: one warp lane per row
constexpr int kSlots64 = 10, kSlots32 = 11;   // slots of the vector blocks
constexpr int kSlotX64 = 8, kSlotInvd = 9;    // x and D^-1 slots
// Jacobi-scaled variant, FP64 block: r wa wb z s p x d sig (sig = a_ii^-1/2)
constexpr int kSlotsS = 9, kSlotXS = 6, kSlotDS = 7, kSlotSigS = 8;
constexpr int kClusterThreads = 256; // CTA size of the cluster path
constexpr int kClusterSize = 8;      // default CTAs per thread-block cluster (portable maximum)

// SELL-C-sigma matrix in the solver's row order (rows permuted within sigma windows when
// sigma > 1; columns renumbered with the same permutation).  Values are A D^-1.
struct DevMatrix {
  int64_t n;
  int64_t nchunks;
  int64_t nslots;
  const int64_t* cptr;   // [nchunks + 1] slot offset of each chunk (multiple of 32)
  const int32_t* col;    // [nslots] column-major within a chunk: slot(base + j*32 + lane)
  // Column dictionary (nullptr when the matrix has more than kColDict distinct offsets):
  // col[s] == row(s) + coff[cidx[s]], row(s) = chunk * 32 + lane of slot s.  Stencil-like
  // matrices have a handful of distinct col - row offsets, so the iteration pass reads one
  // byte per slot instead of four.
  const uint8_t* cidx;   // [nslots]
  const int32_t* coff;   // [kColDict]
  // Offset pattern (pat_k > 0): every row's off-diagonal columns are an ascending subset of
  // row + pat[0..pat_k), pat ascending, and the SELL arrays hold exactly pat_k slots per row
  // (slot p of row i is the entry at column i + pat[p], or a zero with column i when the
  // row has no such entry).  Chunk c's slots start at c * pat_k * 32, and kernels built for
  // the pattern form each column as i + pat[p] (clamped into [0, n)) instead of reading it.
  int32_t pat_k;
  int32_t pat[16];
  const double* val;     // [nslots] a_ij / a_jj
  const float* val32;    // [nslots] same rounded to FP32 (FP32 modes only)
  const double* invd;    // [n] 1 / a_ii
  const float* invd32;   // [n]
  const double* diag;    // [n] a_ii
  const float* diag32;   // [n]
};

// Passes the device state machine can run (one parallel sweep over the rows each).
enum Pass : int32_t {
  P_NONE = 0,
  P_SETUP1,    // r = b - A x ; u = M^-1 r ; partials (b,b) (r,r)
  P_SETUP2,    // w = A u (= Ahat r) ; partials (r,u) (w,u) norm
  P_ITER,      // fused iteration: n = Ahat w ; z q s p x r u w update ; partials
  P_TRUE,      // partial ||b - A x||^2
  P_RR1,       // r = b - A x ; u = M^-1 r ; s = A p ; q = M^-1 s
  P_RR2,       // w = Ahat r ; z = Ahat s ; partials
  P_ZERO_X,    // x = 0
  P_ORES,      // FP32_IR: r64 = b - A x (FP64) ; partials (r64,r64) (b,b)
  P_OINIT,     // FP32_IR: rhs32 = r64 / ||r64|| ; r32 = rhs32 ; u32 = M^-1 r32 ; d32 = 0
  P_OUPD,      // FP32_IR: x += ||r64|| * d32
  P_OUNDO,     // FP32_IR: x -= ||r64_prev|| * d32 (undo a refinement step that did not help)
  P_NORM,      // stopping norm only (after an iteration pass that skipped it)
  P_URES,      // FP32_RU: t = b - A x in FP64 ; r32 = t ; u32 = M^-1 r32 ; s32 = A p32 ;
               //          q32 = M^-1 s32 ; partials (t,t) (b,b)
  P_URR2,      // FP32_RU: w32 = A u32 ; z32 = A q32 ; partials
  P_UFLUSH,    // FP32_RU: x += d32 ; d32 = 0
  P_GAP,       // partials ||(b - A x) - r||^2, ||r||^2 (measured-gap replacement test)
};

// Control states (see control() in solver.cu).
enum State : int32_t {
  // FP64 iteration (also the FP32 modes' fallback): every state below S_O_START
  S_START = 0, S_AFTER_SETUP1, S_AFTER_SETUP2, S_TOP, S_AFTER_ITER, S_AFTER_TRUE, S_AFTER_RR1,
  S_AFTER_RR2, S_FINAL, S_AFTER_FINAL, S_DONE, S_AFTER_NORM, S_AFTER_GAP,
  // FP32_IR
  S_O_START, S_O_AFTER_ORES, S_O_AFTER_ZERO, S_O_AFTER_OINIT, S_I_AFTER_SETUP2, S_I_TOP,
  S_I_AFTER_ITER, S_I_AFTER_RR1, S_I_AFTER_RR2, S_O_AFTER_OUPD, S_O_AFTER_UNDO,
  // FP32_RU
  S_U_START, S_U_AFTER_RES, S_U_AFTER_RR2, S_U_TOP, S_U_AFTER_ITER, S_U_AFTER_FLUSH,
};

// Device-resident control block of one solve.  Read by every CTA at launch start, written
// back by rank 0 at launch end, so a solve can be resumed by a later launch.
struct Ctl {
  int32_t state, pass, status, iter;      // iter: Alg. 2 iterations (inner ones for FP32_IR)
  int32_t inner_iter, outer, rr_count, last_rr_iter;
  int32_t parity, first, exit_now, restart;  // restart: next step starts afresh (beta = 0)
  int32_t restarts, fallback;   // fallback: FP32_IR switched to the FP64 iteration
  int32_t want_rr, rr_valid;    // the next iteration pass accumulates the norm; norm is current
  int32_t norm_return, pad4;    // state to resume after a P_NORM pass
  int32_t stalls, ru_due;       // FP32_RU: reliable updates in a row without progress; this one was due
  double rmax;                  // FP32_RU: largest recursive norm since the last reliable update
  double gamma, gamma_prev, delta, alpha, alpha_prev, beta, norm;
  double inv_gamma, inv_alpha;  // 1 / gamma and 1 / alpha of the last scalars step
  double bnorm, rn, rn_prev, res_true, inner_norm0, inner_target, rr_norm_prev;
  double gamma_ref;             // gamma when the residuals were last measured or replaced
  unsigned long long t_start, t_end;
  double red[4];                           // reduced partials of the last pass
};

struct SysDesc {
  DevMatrix A;
  int32_t precision, norm, rr_period, maxit;
  int32_t inner_maxit, max_outer, nparts, x_zero;  // x_zero: x starts at 0 (skip the A x0 gather)
  int32_t max_restarts, budget;   // budget: iterations this launch may advance (0 = launch's)
  int32_t variant, onchip_slots;  // ppcg_variant; on-chip path: matrix slots of the fullest CTA
  double tol, inner_tol;
  double gap_theta, gap_fall;   // measured-gap replacement (gap_theta 0: off)
  double dmin, dmax;     // extreme diagonal entries (bounds of ||r||^2 / gamma)
  // Matrix-free box stencil (box_g > 0): A = box_cd I + box_co (adjacency of the
  // (2 box_r + 1)^3 box on a box_g^3 grid, truncated at the boundary); box_t holds the
  // four n-row stage arrays (x-sums and y-sums of up to two source vectors).
  int32_t box_g, box_r;
  double box_cd, box_co;
  double* box_t;
  int64_t spin_limit_ns;
  const double* b;       // right-hand side, solver order (plain array)
  // Per-row vectors in chunk-interleaved blocks (for each 32-row chunk, the block's slots
  // of 32 values side by side):
  //   v64: r u wa wb z q s p x invd (FP64 path; FP32_IR keeps its FP64 outer residual in r and
  //        its solution in x, and falls back to the FP64 iteration in this block if needed)
  //   v32: r u wa wb z q s p d invd rhs (FP32_IR inner solve; d is the inner solution)
  double* v64;
  float* v32;
  double* part;          // [2][nparts][4] block partials, double-buffered by pass parity
  Ctl* ctl;
  unsigned* bar;         // grid barrier arrival counter (grid path; zeroed before each launch)
  int32_t* err;          // launch error flag (timeout), zeroed before each launch
};

// Launchers (solver.cu)
cudaError_t launch_grid(const SysDesc* d_desc, int shape, int grid, int budget, cudaStream_t st);
// d_next != nullptr: dynamic schedule over d_list[0..m) (see k_cluster); *d_next must be 0.
// cs: CTAs per cluster (2, 4, 8 or 16; every system of the launch has that plan).
cudaError_t launch_clusters(const SysDesc* d_descs, const int32_t* d_list, const int32_t* d_list_ptr,
                            int nclusters, int budget, cudaStream_t st, bool spread = false,
                            int32_t* d_next = nullptr, int32_t m = 0, int cs = 8);
// On-chip path, clusters of nc = 8 or 16 CTAs (16: non-portable, where the device allows).
cudaError_t launch_onchip(const SysDesc* d_descs, const int32_t* d_list, const int32_t* d_list_ptr,
                          int nclusters, int budget, size_t smem, int nc, cudaStream_t st);
size_t onchip_smem_bytes(int64_t nchunks, int64_t slots, int nc);   // dynamic shared memory per CTA
size_t onchip_smem_limit(int device);                               // largest the device allows
bool onchip_cluster_fits(int nc, size_t smem);                      // can one such cluster run
int grid_shape_count();        // SELL/CSR plans: shapes [0, grid_shape_count())
int grid_box_shape_first();    // matrix-free box plans: shapes first + [0, count)
int grid_box_shape_count();
// The default SELL shape for a column source (PPCG_COLS_SELL, PPCG_COLS_DICT or
// PPCG_COLS_PATTERN) and precision (the FP32 forms run more warps per CTA).
// streaming: the system's FP64 vector block exceeds half the L2 (the own-entry prefetch pays)
int grid_default_shape(int cols, bool fp32, bool streaming);
int grid_shape_cols(int shape);   // the column source (PPCG_COLS_*) a SELL shape's kernel reads
int grid_threads(int shape);
int grid_blocks_for_device(int device, int shape);
int max_active_clusters(int device, int cs = 8);   // 0 when clusters of cs CTAs cannot run
cudaError_t launch_barrier_selftest(unsigned* bar, int32_t* err, int32_t* out, int grid,
                                    int drop_rank, int64_t limit_ns, cudaStream_t st);

// Conversion (convert.cu)
constexpr int kColDict = 255;   // largest column dictionary (a one-byte index)

struct SellBuild {
  int64_t nchunks = 0, nslots = 0;
  int32_t sigma = 1;
  double padding = 0.0;   // padded slots / off-diagonal nonzeros
  double seconds = 0.0;   // conversion wall time
  double dmin = 0.0, dmax = 0.0;   // extreme diagonal entries
  int64_t onchip_slots = 0;        // SELL slots of the fullest CTA when chunk c goes to CTA c % 8
  int64_t onchip_slots16 = 0;      // the same for clusters of 16 CTAs
  int32_t col_dict = 0;            // distinct col - row offsets in the dictionary (0: none)
  int32_t pattern_k = 0;           // offsets of the offset pattern (0: none; see DevMatrix)
};
constexpr int kPatMax = 16;      // largest offset pattern
ppcg_status convert_csr_to_sell(int64_t n, int64_t nnz, const int64_t* d_rp, const int32_t* d_col,
                                const double* d_val, int32_t sigma_req, bool want_fp32, bool sym_scale,
                                cudaStream_t st, std::vector<void*>& allocs, SellBuild* out,
                                DevMatrix* A, int32_t** d_perm_out);

// Is the (validated, device) CSR a constant-coefficient box stencil cd I + co (box adjacency)
// on a g^3 grid, rows in grid order?  Synchronises st.
bool detect_box_stencil(int64_t n, int64_t nnz, const int64_t* d_rp, const int32_t* d_col, const double* d_val,
                        cudaStream_t st, int32_t* g, int32_t* r, double* cd, double* co);

void set_error(const char* fmt, ...);

// NVTX range over a host-side scope (create, enqueue of a solve or batch, server admission
// and epochs), for timeline profilers; header-only NVTX 3, no cost when no tool listens.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device memory of handles comes from a library-owned stream-ordered pool per device (no
// device-wide synchronisation on allocation or release; freed blocks stay in the pool).
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st);
void pool_free(void* p, cudaStream_t st);

}  // namespace ppcg
