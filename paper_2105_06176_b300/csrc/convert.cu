// CSR -> SELL-C-sigma conversion with the Jacobi diagonal (Sec. V-A: CSR input, Jacobi
// preconditioner M = diag(A)).  Runs once per handle inside ppcg_create.
//
// The solver keeps the matrix column-scaled, Ahat = A D^-1 (or, for the Jacobi-scaled
// variant, symmetrically scaled, D^-1/2 A D^-1/2, with the same unit diagonal), so that the preconditioner
// apply and the SpMV of Alg. 2 (m = M^-1 w; n = A m) become one product
// n = Ahat w with no per-iteration multiply by D^-1 inside the gather.  The scaling divides
// (a_ij / a_jj), so every diagonal entry of Ahat is exactly 1.0: the SELL arrays hold the
// off-diagonal entries only and the kernels add the diagonal term (w_i, or a_ii v_i for
// A v) exactly, as the first term of each row sum.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

namespace ppcg {

namespace {

enum : int32_t { F_ARG = 1, F_NOT_SPD = 2 };

// One thread per row: validate the row, extract the diagonal, record the row length; also
// the extreme diagonal entries (for positive doubles the order of the bit patterns is the
// numeric order, so integer min / max serve; one atomic pair per warp).
__global__ void k_rows(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                       const int32_t* __restrict__ col, const double* __restrict__ val,
                       double* __restrict__ diag, double* __restrict__ invd,
                       int32_t* __restrict__ rowlen, int32_t* flags, unsigned long long* dminmax) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long lo = ~0ull, hi = 0ull;
  if (i < n) {
    int64_t a = rp[i], e = rp[i + 1];
    int32_t f = 0;
    if (a < 0 || e < a || e > nnz || (i == 0 && a != 0) || (i == n - 1 && e != nnz)) {
      f |= F_ARG;
      e = a;
    }
    if (e - a > INT32_MAX) { f |= F_ARG; e = a; }
    double d = 0.0;
    bool found = false;
    int32_t off = 0;
    for (int64_t k = a; k < e; k++) {
      int32_t c = col[k];
      if (c < 0 || c >= n) f |= F_ARG;
      if (c == i) { d += val[k]; found = true; } else { off++; }
    }
    if (!found || !(d > 0.0)) f |= F_NOT_SPD;
    rowlen[i] = off;          // off-diagonal entries of the row
    diag[i] = d;
    invd[i] = found && d > 0.0 ? 1.0 / d : 0.0;
    if (f) atomicOr(flags, f);
    if (found && d > 0.0) lo = hi = (unsigned long long)__double_as_longlong(d);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) { atomicMin(dminmax, lo); atomicMax(dminmax + 1, hi); }
}

// One thread per (chunk row): write the row's off-diagonal slots, column-major inside its
// chunk, in CSR order.
__global__ void k_fill(int64_t n, int64_t nchunks, const int64_t* __restrict__ rp,
                       const int32_t* __restrict__ col, const double* __restrict__ val,
                       const double* __restrict__ diag, const int32_t* __restrict__ rowlen,
                       const int32_t* __restrict__ perm, const int32_t* __restrict__ iperm,
                       const int64_t* __restrict__ cptr, int32_t* __restrict__ scol,
                       double* __restrict__ sval, float* __restrict__ sval32, int sym) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t c = t / kChunk;
  int lane = (int)(t % kChunk);
  if (c >= nchunks) return;
  int64_t i = c * kChunk + lane;
  int64_t base = cptr[c];
  int len = (int)((cptr[c + 1] - base) / kChunk);
  int64_t o = i < n ? (perm ? perm[i] : i) : 0;
  int64_t a = i < n ? rp[o] : 0;
  int64_t e = i < n ? rp[o + 1] : 0;
  int j = 0;
  for (int64_t k = a; k < e; k++) {
    int32_t oc = col[k];
    if (oc == o) continue;                       // diagonal: implicit, exactly 1 after scaling
    int64_t slot = base + (int64_t)j * kChunk + lane;
    // A D^-1 (column scaling), or D^-1/2 A D^-1/2 for the symmetrically scaled variant
    double v = sym ? val[k] / (sqrt(diag[o]) * sqrt(diag[oc])) : val[k] / diag[oc];
    scol[slot] = iperm ? iperm[oc] : oc;
    sval[slot] = v;
    if (sval32) sval32[slot] = (float)v;
    j++;
  }
  for (; j < len; j++) {                         // padding: a zero that gathers the row's own entry
    int64_t slot = base + (int64_t)j * kChunk + lane;
    scol[slot] = (int32_t)(i < n ? i : n - 1);
    sval[slot] = 0.0;
    if (sval32) sval32[slot] = 0.0f;
  }
}

// Column dictionary.  The distinct offsets col - row of the SELL slots are collected in an
// open-addressing table of kDictTable entries (kDictEmpty marks a free entry); then every
// slot gets the one-byte index of its offset.  Collection stops (overflow) once more than
// kColDict offsets appear: unstructured matrices keep their 4-byte columns.
constexpr int kDictTable = 1024;
constexpr int32_t kDictEmpty = INT32_MIN;

__device__ __forceinline__ int dict_probe(int32_t* table, int32_t key, bool insert, int32_t* count,
                                          int32_t* overflow, int32_t limit = kColDict) {
  const uint32_t h = (uint32_t)key * 2654435761u;
  for (int probe = 0; probe < kDictTable; probe++) {
    const int pos = (int)((h + (uint32_t)probe) & (kDictTable - 1));
    const int32_t cur = ((volatile int32_t*)table)[pos];
    if (cur == key) return pos;
    if (cur != kDictEmpty) continue;
    if (!insert || *(volatile int32_t*)overflow) return -1;
    const int32_t prev = atomicCAS(table + pos, kDictEmpty, key);
    if (prev == kDictEmpty) {
      if (atomicAdd(count, 1) >= limit) atomicExch(overflow, 1);
      return pos;
    }
    if (prev == key) return pos;
  }
  atomicExch(overflow, 1);
  return -1;
}

// One thread per (chunk, lane), as k_fill: insert the offsets of the lane's slots (pass 0),
// or write each slot's dictionary index (pass 1, after the table is final).
__global__ void k_dict(int64_t nchunks, const int64_t* __restrict__ cptr, const int32_t* __restrict__ scol,
                       int32_t* table, int32_t* count, int32_t* overflow, const uint8_t* __restrict__ pos2idx,
                       uint8_t* __restrict__ cidx) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t c = t / kChunk;
  const int lane = (int)(t % kChunk);
  if (c >= nchunks) return;
  const int64_t i = c * kChunk + lane;
  const int64_t base = cptr[c];
  const int len = (int)((cptr[c + 1] - base) / kChunk);
  for (int j = 0; j < len; j++) {
    const int64_t slot = base + (int64_t)j * kChunk + lane;
    const int32_t key = (int32_t)((int64_t)scol[slot] - i);
    if (!cidx) {
      if (dict_probe(table, key, true, count, overflow) < 0) return;
    } else {
      const int pos = dict_probe(table, key, false, count, overflow);
      cidx[slot] = pos < 0 ? 0 : pos2idx[pos];
    }
  }
}

// Offset pattern, first pass.  One thread per row: insert the row's off-diagonal offsets
// col - row into the table (overflow beyond kPatMax distinct offsets), and flag a row whose
// off-diagonal offsets do not ascend in CSR order (then the pattern order would not be the
// row's summation order).
__global__ void k_pat_offsets(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              int32_t* table, int32_t* count, int32_t* overflow, int32_t* unsorted) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t prev = INT64_MIN;
  for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
    const int64_t c = col[k];
    if (c == i) continue;
    const int64_t off = c - i;
    if (off <= prev) atomicExch(unsorted, 1);
    prev = off;
    if (dict_probe(table, (int32_t)off, true, count, overflow, kPatMax) < 0) return;
  }
}

// Offset pattern, fill.  One thread per (chunk, lane): the row's pat_k slots, slot p holding
// the row's entry at column i + pat[p] (scaled as in k_fill), or a zero with column i where
// the row has no such entry (rows past n: zeros with column n - 1).  Rows are in CSR order.
__global__ void k_fill_pat(int64_t n, int64_t nchunks, const int64_t* __restrict__ rp,
                           const int32_t* __restrict__ col, const double* __restrict__ val,
                           const double* __restrict__ diag, const int32_t* __restrict__ pat, int K,
                           int32_t* __restrict__ scol, double* __restrict__ sval, float* __restrict__ sval32,
                           int sym) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t c = t / kChunk;
  const int lane = (int)(t % kChunk);
  if (c >= nchunks) return;
  const int64_t i = c * kChunk + lane;
  const int64_t base = c * (int64_t)K * kChunk + lane;
  const int32_t self = (int32_t)(i < n ? i : n - 1);
  for (int p = 0; p < K; p++) {
    scol[base + (int64_t)p * kChunk] = self;
    sval[base + (int64_t)p * kChunk] = 0.0;
    if (sval32) sval32[base + (int64_t)p * kChunk] = 0.0f;
  }
  if (i >= n) return;
  int p = 0;
  for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
    const int32_t oc = col[k];
    if (oc == i) continue;
    const int64_t off = (int64_t)oc - i;
    while (p < K && pat[p] != off) p++;            // offsets ascend in the row and in pat
    if (p == K) return;                            // cannot happen after k_pat_offsets
    const double v = sym ? val[k] / (sqrt(diag[i]) * sqrt(diag[oc])) : val[k] / diag[oc];
    const int64_t slot = base + (int64_t)p * kChunk;
    scol[slot] = oc;
    sval[slot] = v;
    if (sval32) sval32[slot] = (float)v;
    p++;
  }
}

// Vectors in solver order, plus FP32 copies.
__global__ void k_permute_diag(int64_t n, const int32_t* __restrict__ perm,
                               const double* __restrict__ diag, const double* __restrict__ invd,
                               double* __restrict__ sdiag, double* __restrict__ sinvd,
                               float* __restrict__ sdiag32, float* __restrict__ sinvd32) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t o = perm ? perm[i] : i;
  double d = diag[o], id = invd[o];
  sdiag[i] = d;
  sinvd[i] = id;
  if (sdiag32) { sdiag32[i] = (float)d; sinvd32[i] = (float)id; }
}

template <typename T>
cudaError_t dalloc(T** p, size_t count, std::vector<void*>& allocs, cudaStream_t st) {
  cudaError_t e = pool_alloc((void**)p, std::max<size_t>(count, 1) * sizeof(T), st);
  if (e == cudaSuccess) allocs.push_back(*p);
  return e;
}

// Stable order of the rows of one window by decreasing length: a counting sort over the
// window's length histogram (row lengths are small for sparse matrices), with a comparison
// sort as the fallback for windows holding very long rows.
void sort_window(const std::vector<int32_t>& len, int64_t w0, int64_t w1, int32_t* out,
                 std::vector<int64_t>& hist) {
  int32_t mx = 0;
  for (int64_t i = w0; i < w1; i++) mx = std::max(mx, len[i]);
  if (mx > 4096) {
    std::iota(out, out + (w1 - w0), (int32_t)w0);
    std::stable_sort(out, out + (w1 - w0), [&](int32_t a, int32_t b) { return len[a] > len[b]; });
    return;
  }
  hist.assign(mx + 2, 0);
  for (int64_t i = w0; i < w1; i++) hist[mx - len[i] + 1]++;          // bucket 0 = longest
  for (int32_t k = 1; k <= mx + 1; k++) hist[k] += hist[k - 1];        // start offsets
  for (int64_t i = w0; i < w1; i++) out[hist[mx - len[i]]++] = (int32_t)i;
}

// Slots of SELL-C-sigma for the given row lengths: rows sorted by decreasing length inside
// windows of sigma rows (stable), chunks of 32 consecutive sorted rows padded to their
// longest row.  Returns the slot count; fills perm and cptr when asked.
int64_t sell_slots(const std::vector<int32_t>& len, int64_t sigma, std::vector<int32_t>* perm,
                   std::vector<int64_t>* cptr) {
  const int64_t n = (int64_t)len.size();
  const int64_t nchunks = (n + kChunk - 1) / kChunk;
  std::vector<int32_t> p;
  std::vector<int64_t> hist;
  if (sigma > 1) {
    p.resize(n);
    for (int64_t w0 = 0; w0 < n; w0 += sigma) sort_window(len, w0, std::min(n, w0 + sigma), p.data() + w0, hist);
  }
  if (cptr) cptr->assign(nchunks + 1, 0);
  int64_t slots = 0;
  for (int64_t c = 0; c < nchunks; c++) {
    int32_t mx = 0;
    for (int64_t i = c * kChunk; i < std::min(n, (c + 1) * kChunk); i++)
      mx = std::max(mx, len[sigma > 1 ? p[i] : i]);
    slots += (int64_t)mx * kChunk;
    if (cptr) (*cptr)[c + 1] = slots;
  }
  if (perm) *perm = std::move(p);
  return slots;
}

// One thread per row: does the row hold exactly the in-grid cells of its (2R+1)^3 box in
// ascending column order, with value cd on the diagonal and co elsewhere?
__global__ void k_box_check(int64_t n, int32_t g, int32_t R, const int64_t* __restrict__ rp,
                            const int32_t* __restrict__ col, const double* __restrict__ val, double cd,
                            double co, int32_t* bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t x = (int32_t)(i % g), y = (int32_t)((i / g) % g), z = (int32_t)(i / ((int64_t)g * g));
  auto span = [&](int32_t c) { return min(c, R) + min(g - 1 - c, R) + 1; };
  const int64_t a = rp[i], e = rp[i + 1];
  if (e - a != (int64_t)span(x) * span(y) * span(z)) { atomicOr(bad, 1); return; }
  int64_t prev = -1;
  for (int64_t k = a; k < e; k++) {
    const int64_t j = col[k];
    const int32_t jx = (int32_t)(j % g), jy = (int32_t)((j / g) % g), jz = (int32_t)(j / ((int64_t)g * g));
    const bool in = abs(jx - x) <= R && abs(jy - y) <= R && abs(jz - z) <= R;
    const double want = j == i ? cd : co;
    if (j <= prev || !in || val[k] != want) { atomicOr(bad, 1); return; }
    prev = j;
  }
}

}  // namespace

bool detect_box_stencil(int64_t n, int64_t nnz, const int64_t* d_rp, const int32_t* d_col, const double* d_val,
                        cudaStream_t st, int32_t* g_out, int32_t* r_out, double* cd_out, double* co_out) {
  if (n < 27) return false;
  const int32_t g = (int32_t)std::llround(std::cbrt((double)n));
  if ((int64_t)g * g * g != n) return false;
  // row 0 is a corner: (R + 1)^3 entries, the diagonal first
  int64_t rp01[2];
  if (cudaMemcpyAsync(rp01, d_rp, sizeof(rp01), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); return false; }
  const int64_t cnt = rp01[1] - rp01[0];
  const int32_t R = (int32_t)std::llround(std::cbrt((double)cnt)) - 1;
  if (R < 1 || R > 3 || (int64_t)(R + 1) * (R + 1) * (R + 1) != cnt || g < 2 * R + 1) return false;
  int32_t c2[2];
  double v2[2];
  if (cudaMemcpyAsync(c2, d_col + rp01[0], sizeof(c2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(v2, d_val + rp01[0], sizeof(v2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); return false; }
  if (c2[0] != 0 || c2[1] == 0) return false;
  const double cd = v2[0], co = v2[1];
  if (!(cd > 0.0) || !(co != 0.0)) return false;
  int32_t* d_bad = nullptr;
  if (pool_alloc((void**)&d_bad, sizeof(int32_t), st) != cudaSuccess) { cudaGetLastError(); return false; }
  cudaMemsetAsync(d_bad, 0, sizeof(int32_t), st);
  const int tb = 256;
  k_box_check<<<(unsigned)((n + tb - 1) / tb), tb, 0, st>>>(n, g, R, d_rp, d_col, d_val, cd, co, d_bad);
  int32_t bad = 1;
  cudaMemcpyAsync(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  const bool ok = cudaStreamSynchronize(st) == cudaSuccess && bad == 0;
  cudaGetLastError();
  pool_free(d_bad, st);
  (void)nnz;
  if (!ok) return false;
  *g_out = g;
  *r_out = R;
  *cd_out = cd;
  *co_out = co;
  return true;
}

// Build A's column dictionary on the device; leaves A->cidx = nullptr (and returns 0) when
// the matrix has more than kColDict distinct offsets or PPCG_COL_DICT=0 is set.  Returns the
// dictionary size, or -1 when a device allocation failed.  Synchronises st.
int build_col_dict(DevMatrix* A, std::vector<void*>& allocs, cudaStream_t st) {
  A->cidx = nullptr;
  A->coff = nullptr;
  if (const char* e = getenv("PPCG_COL_DICT")) if (e[0] == '0') return 0;   // diagnostic knob
  if (A->nslots == 0) return 0;
  int32_t* d_tab = nullptr;   // table, count, overflow
  if (pool_alloc((void**)&d_tab, (kDictTable + 2) * sizeof(int32_t), st) != cudaSuccess) { cudaGetLastError(); return -1; }
  std::vector<int32_t> h(kDictTable + 2, kDictEmpty);
  h[kDictTable] = 0;
  h[kDictTable + 1] = 0;
  cudaMemcpyAsync(d_tab, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  const int tb = 256;
  const int64_t threads = A->nchunks * kChunk;
  const unsigned blocks = (unsigned)((threads + tb - 1) / tb);
  k_dict<<<blocks, tb, 0, st>>>(A->nchunks, A->cptr, A->col, d_tab, d_tab + kDictTable, d_tab + kDictTable + 1,
                                nullptr, nullptr);
  cudaMemcpyAsync(h.data(), d_tab, h.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  int size = 0;
  bool oom = false;
  uint8_t* d_cidx = nullptr;
  int32_t* d_coff = nullptr;
  uint8_t* d_pos2idx = nullptr;
  if (cudaStreamSynchronize(st) == cudaSuccess && h[kDictTable + 1] == 0 && h[kDictTable] <= kColDict) {
    std::vector<uint8_t> pos2idx(kDictTable, 0);
    std::vector<int32_t> coff(kColDict, 0);
    for (int pos = 0; pos < kDictTable; pos++)
      if (h[pos] != kDictEmpty) { pos2idx[pos] = (uint8_t)size; coff[size++] = h[pos]; }
    if (dalloc(&d_cidx, (size_t)A->nslots, allocs, st) == cudaSuccess &&
        dalloc(&d_coff, (size_t)kColDict, allocs, st) == cudaSuccess &&
        pool_alloc((void**)&d_pos2idx, kDictTable, st) == cudaSuccess) {
      cudaMemcpyAsync(d_coff, coff.data(), kColDict * sizeof(int32_t), cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(d_pos2idx, pos2idx.data(), kDictTable, cudaMemcpyHostToDevice, st);
      k_dict<<<blocks, tb, 0, st>>>(A->nchunks, A->cptr, A->col, d_tab, d_tab + kDictTable,
                                    d_tab + kDictTable + 1, d_pos2idx, d_cidx);
      if (cudaStreamSynchronize(st) == cudaSuccess && cudaGetLastError() == cudaSuccess) {
        A->cidx = d_cidx;
        A->coff = d_coff;
      } else {
        size = 0;
      }
    } else {
      size = 0;
      oom = true;
    }
  }
  cudaGetLastError();
  if (d_pos2idx) pool_free(d_pos2idx, st);
  pool_free(d_tab, st);
  if (oom) return -1;
  return A->cidx ? size : 0;
}

ppcg_status convert_csr_to_sell(int64_t n, int64_t nnz, const int64_t* d_rp, const int32_t* d_col,
                                const double* d_val, int32_t sigma_req, bool want_fp32, bool sym_scale,
                                cudaStream_t st, std::vector<void*>& allocs, SellBuild* out,
                                DevMatrix* A, int32_t** d_perm_out) {
  auto t0 = std::chrono::steady_clock::now();
  std::vector<void*> tmp;
  auto free_tmp = [&]() { for (void* p : tmp) pool_free(p, st); tmp.clear(); };
  double *d_diag0 = nullptr, *d_invd0 = nullptr;
  int32_t *d_len = nullptr, *d_flags = nullptr;
  unsigned long long* d_mm = nullptr;
  cudaError_t e = cudaSuccess;
  if ((e = dalloc(&d_diag0, n, tmp, st)) || (e = dalloc(&d_invd0, n, tmp, st)) ||
      (e = dalloc(&d_len, n, tmp, st)) || (e = dalloc(&d_flags, 1, tmp, st)) ||
      (e = dalloc(&d_mm, 2, tmp, st))) {
    free_tmp();
    set_error("ppcg_create: device allocation failed: %s", cudaGetErrorString(e));
    return PPCG_ERR_OOM;
  }
  cudaMemsetAsync(d_flags, 0, sizeof(int32_t), st);
  cudaMemsetAsync(d_mm, 0xff, sizeof(unsigned long long), st);        // min: all ones
  cudaMemsetAsync(d_mm + 1, 0, sizeof(unsigned long long), st);       // max: 0
  const int tb = 256;
  k_rows<<<(unsigned)((n + tb - 1) / tb), tb, 0, st>>>(n, nnz, d_rp, d_col, d_val, d_diag0, d_invd0,
                                                       d_len, d_flags, d_mm);
  int32_t flags = 0;
  unsigned long long mm[2] = {0, 0};
  std::vector<int32_t> len(n);
  cudaMemcpyAsync(&flags, d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(mm, d_mm, sizeof(mm), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(len.data(), d_len, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
    free_tmp();
    set_error("ppcg_create: %s", cudaGetErrorString(e));
    return PPCG_ERR_CUDA;
  }
  if (flags & F_ARG) { free_tmp(); set_error("ppcg_create: malformed CSR (row_ptr or column index)"); return PPCG_ERR_ARG; }
  if (flags & F_NOT_SPD) { free_tmp(); set_error("ppcg_create: missing or non-positive diagonal entry"); return PPCG_ERR_NOT_SPD; }

  // Offset pattern (see DevMatrix): stencil-like matrices whose rows all draw their
  // off-diagonal columns, in ascending order, from at most kPatMax offsets.  Taken when its
  // slots (pat_k per row, zeros where a row lacks a neighbour) are at most 1.25x the slots
  // of sigma = 1 SELL: a pattern slot carries no column bytes, a SELL slot four.
  std::vector<int32_t> pat;
  const char* no_dict = getenv("PPCG_COL_DICT");                    // diagnostic knobs: "0" = off
  const char* no_pat = getenv("PPCG_COL_PAT");
  if ((sigma_req <= 1) && !(no_dict && no_dict[0] == '0') && !(no_pat && no_pat[0] == '0') && nnz > n) {
    int32_t* d_tab = nullptr;   // table, count, overflow, unsorted
    if ((e = dalloc(&d_tab, kDictTable + 3, tmp, st)) != cudaSuccess) {
      free_tmp();
      set_error("ppcg_create: device allocation failed: %s", cudaGetErrorString(e));
      return PPCG_ERR_OOM;
    }
    std::vector<int32_t> h(kDictTable + 3, kDictEmpty);
    h[kDictTable] = h[kDictTable + 1] = h[kDictTable + 2] = 0;
    cudaMemcpyAsync(d_tab, h.data(), h.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    k_pat_offsets<<<(unsigned)((n + tb - 1) / tb), tb, 0, st>>>(n, d_rp, d_col, d_tab, d_tab + kDictTable,
                                                                d_tab + kDictTable + 1, d_tab + kDictTable + 2);
    cudaMemcpyAsync(h.data(), d_tab, h.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
      free_tmp();
      set_error("ppcg_create: %s", cudaGetErrorString(e));
      return PPCG_ERR_CUDA;
    }
    if (h[kDictTable + 1] == 0 && h[kDictTable + 2] == 0 && h[kDictTable] >= 1 && h[kDictTable] <= kPatMax) {
      for (int k = 0; k < kDictTable; k++)
        if (h[k] != kDictEmpty) pat.push_back(h[k]);
      std::sort(pat.begin(), pat.end());
      const int64_t pat_slots = (int64_t)pat.size() * kChunk * ((n + kChunk - 1) / kChunk);
      if ((double)pat_slots > 1.25 * (double)sell_slots(len, 1, nullptr, nullptr)) pat.clear();
    }
  }

  // sigma autotune.  Sorting rows by length within a window of sigma > C rows cuts the
  // padding (and with it the padded slots' bytes and FMAs), but it also scatters the rows of
  // a chunk over the window, so the 32 lanes of a warp gather from less related rows and the
  // gathers touch more L1/L2 sectors.  Model per iteration: padded slots x (value + column
  // bytes) + a gather penalty per off-diagonal nonzero, in bytes of equivalent HBM traffic:
  // 1.4 at sigma = 64, 3.0 at 128, 4.2 at 256 (fitted to the FP64 and FP32_RU solve times of
  // a 4M-point random-geometric-graph Laplacian, 14.9 nonzeros per row: padding 52% / 30% /
  // 17% / 9%, FP64 289 / 278 / 279 / 280 ms, FP32_RU 235 / 229 / 235 / 247 ms) and 16 at
  // 2048 (where sigma = 1 had run 17% (FP64) and 27% (FP32) faster).  The smallest cost wins.
  int64_t sigma = sigma_req;
  if (!pat.empty()) {
    sigma = 1;
  } else if (sigma_req <= 0) {
    const int64_t cands[] = {1, 64, 128, 256, 2048};
    const double penalty[] = {0.0, 1.4, 3.0, 4.2, 16.0};
    const double slot_bytes = want_fp32 ? 8.0 : 12.0;
    int64_t offdiag = 0;
    for (int64_t i = 0; i < n; i++) offdiag += len[i];
    double best = 0.0;
    for (int k = 0; k < 5; k++) {
      const double cost = (double)sell_slots(len, cands[k], nullptr, nullptr) * slot_bytes + penalty[k] * (double)offdiag;
      if (k == 0 || cost < best) { best = cost; sigma = cands[k]; }
    }
  }
  std::vector<int32_t> perm;
  std::vector<int64_t> cptr;
  const int K = (int)pat.size();
  int64_t nslots = 0;
  if (K > 0) {                     // pat_k slots in every row
    const int64_t nch = (n + kChunk - 1) / kChunk;
    cptr.resize(nch + 1);
    for (int64_t c = 0; c <= nch; c++) cptr[c] = c * K * kChunk;
    nslots = nch * K * kChunk;
  } else {
    nslots = sell_slots(len, sigma, &perm, &cptr);
  }
  const int64_t nchunks = (int64_t)cptr.size() - 1;

  int64_t* d_cptr = nullptr; int32_t* d_scol = nullptr; double* d_sval = nullptr; float* d_sval32 = nullptr;
  double *d_sdiag = nullptr, *d_sinvd = nullptr; float *d_sdiag32 = nullptr, *d_sinvd32 = nullptr;
  int32_t *d_perm = nullptr, *d_iperm = nullptr;
  if ((e = dalloc(&d_cptr, nchunks + 1, allocs, st)) || (e = dalloc(&d_scol, nslots, allocs, st)) ||
      (e = dalloc(&d_sval, nslots, allocs, st)) || (e = dalloc(&d_sdiag, n, allocs, st)) ||
      (e = dalloc(&d_sinvd, n, allocs, st)) ||
      (want_fp32 && ((e = dalloc(&d_sval32, nslots, allocs, st)) || (e = dalloc(&d_sdiag32, n, allocs, st)) ||
                     (e = dalloc(&d_sinvd32, n, allocs, st))))) {
    free_tmp();
    set_error("ppcg_create: device allocation failed: %s", cudaGetErrorString(e));
    return PPCG_ERR_OOM;
  }
  if (!perm.empty()) {
    std::vector<int32_t> iperm(n);
    for (int64_t i = 0; i < n; i++) iperm[perm[i]] = (int32_t)i;
    if ((e = dalloc(&d_perm, n, allocs, st)) || (e = dalloc(&d_iperm, n, tmp, st))) {
      free_tmp();
      set_error("ppcg_create: device allocation failed: %s", cudaGetErrorString(e));
      return PPCG_ERR_OOM;
    }
    cudaMemcpyAsync(d_perm, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_iperm, iperm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    // keep iperm alive until the copies and the fill kernel complete (sync below)
    cudaMemcpyAsync(d_cptr, cptr.data(), (nchunks + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    int64_t threads = nchunks * kChunk;
    k_fill<<<(unsigned)((threads + tb - 1) / tb), tb, 0, st>>>(n, nchunks, d_rp, d_col, d_val, d_diag0,
                                                               d_len, d_perm, d_iperm, d_cptr, d_scol,
                                                               d_sval, d_sval32, sym_scale ? 1 : 0);
    k_permute_diag<<<(unsigned)((n + tb - 1) / tb), tb, 0, st>>>(n, d_perm, d_diag0, d_invd0, d_sdiag,
                                                                 d_sinvd, d_sdiag32, d_sinvd32);
    e = cudaStreamSynchronize(st);
  } else {
    cudaMemcpyAsync(d_cptr, cptr.data(), (nchunks + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st);
    int64_t threads = nchunks * kChunk;
    if (K > 0) {
      int32_t* d_pat = nullptr;
      if ((e = dalloc(&d_pat, K, tmp, st)) != cudaSuccess) {
        free_tmp();
        set_error("ppcg_create: device allocation failed: %s", cudaGetErrorString(e));
        return PPCG_ERR_OOM;
      }
      cudaMemcpyAsync(d_pat, pat.data(), K * sizeof(int32_t), cudaMemcpyHostToDevice, st);
      k_fill_pat<<<(unsigned)((threads + tb - 1) / tb), tb, 0, st>>>(n, nchunks, d_rp, d_col, d_val, d_diag0,
                                                                     d_pat, K, d_scol, d_sval, d_sval32,
                                                                     sym_scale ? 1 : 0);
    } else {
      k_fill<<<(unsigned)((threads + tb - 1) / tb), tb, 0, st>>>(n, nchunks, d_rp, d_col, d_val, d_diag0,
                                                                 d_len, nullptr, nullptr, d_cptr, d_scol,
                                                                 d_sval, d_sval32, sym_scale ? 1 : 0);
    }
    k_permute_diag<<<(unsigned)((n + tb - 1) / tb), tb, 0, st>>>(n, nullptr, d_diag0, d_invd0, d_sdiag,
                                                                 d_sinvd, d_sdiag32, d_sinvd32);
    e = cudaStreamSynchronize(st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  free_tmp();
  if (e != cudaSuccess) {
    set_error("ppcg_create: conversion failed: %s", cudaGetErrorString(e));
    return PPCG_ERR_CUDA;
  }
  A->n = n;
  A->nchunks = nchunks;
  A->nslots = nslots;
  A->cptr = d_cptr;
  A->col = d_scol;
  A->cidx = nullptr;
  A->coff = nullptr;
  A->pat_k = K;
  for (int k = 0; k < kPatMax; k++) A->pat[k] = k < K ? pat[k] : 0;
  A->val = d_sval;
  A->val32 = d_sval32;
  A->invd = d_sinvd;
  A->invd32 = d_sinvd32;
  A->diag = d_sdiag;
  A->diag32 = d_sdiag32;
  *d_perm_out = d_perm;
  out->nchunks = nchunks;
  out->nslots = nslots;
  {
    int64_t per[16] = {0};
    for (int64_t c = 0; c < nchunks; c++) per[c % 16] += cptr[c + 1] - cptr[c];
    out->onchip_slots16 = *std::max_element(per, per + 16);
    int64_t per8[8];
    for (int r = 0; r < 8; r++) per8[r] = per[r] + per[r + 8];   // c % 8 == r  <=>  c % 16 in {r, r + 8}
    out->onchip_slots = *std::max_element(per8, per8 + 8);
  }
  out->pattern_k = K;
  out->col_dict = K > 0 ? 0 : build_col_dict(A, allocs, st);   // the pattern needs no dictionary
  if (out->col_dict < 0) {
    set_error("ppcg_create: out of device memory for the column dictionary");
    return PPCG_ERR_OOM;
  }
  out->sigma = (int32_t)sigma;
  out->padding = nnz > n ? (double)(nslots - (nnz - n)) / (double)(nnz - n) : 0.0;
  std::memcpy(&out->dmin, &mm[0], sizeof(double));
  std::memcpy(&out->dmax, &mm[1], sizeof(double));
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return PPCG_OK;
}

}  // namespace ppcg
