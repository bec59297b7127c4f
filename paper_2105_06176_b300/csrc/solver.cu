// Device side of the pipelined PCG solver: Algorithm 2 of Tiwari & Vadhiyar (arXiv
// 2105.06176, Sec. III-B) with the Jacobi preconditioner (Sec. V-A), run as a resumable
// state machine inside one persistent launch.
//
// Every CTA of a group (the whole grid, or one thread-block cluster) runs the same control
// logic on the same reduced scalars, so all CTAs take the same branch with no broadcast.
// One "pass" is one sweep over the system's rows in SELL-C-sigma order (one warp per
// 32-row chunk, one lane per row); passes are separated by a group barrier.  The hot pass,
// P_ITER, is the whole iteration of Alg. 2 for its rows:
//     n_i  = A M^-1 w_i  = Ahat w_i           (preconditioner and SpMV of the previous step)
//     z = n + beta z;  q = m + beta q;  s = w + beta s;  p = u + beta p     (vector updates)
//     x += alpha p;    r -= alpha s;    u -= alpha q;    w -= alpha z
//     block partials of (r,u), (w,u) and the stopping norm                  (dot products)
// with w double-buffered (other CTAs still gather the old w), and alpha/beta formed after
// the barrier from the partials in a fixed order.
#include <cstdio>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "internal.h"

namespace ppcg {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ---------------------------------------------------------------------------- groups --

// Whole-grid group (cooperative launch: all CTAs are co-resident).  The barrier is a
// monotone arrival counter zeroed before the launch; each wait is bounded in time.
struct GridGroup {
  static constexpr bool kCluster = false;
  unsigned* bar;
  int32_t* err;
  long long limit_ns;
  unsigned epoch;
  __device__ int rank() const { return blockIdx.x; }
  __device__ int size() const { return gridDim.x; }
  __device__ bool sync() {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
      int good = 1;
      epoch++;
      const unsigned target = epoch * gridDim.x;
      __threadfence();
      atomicAdd(bar, 1u);
      const unsigned long long t0 = globaltimer();
      unsigned spins = 0;
      for (;;) {
        unsigned v = ld_acquire_gpu(bar);
        if ((int)(v - target) >= 0) break;
        if (*(volatile int32_t*)err != 0) { good = 0; break; }
        if ((++spins & 63u) == 0 && (long long)(globaltimer() - t0) > limit_ns) {
          atomicCAS(err, 0, (int32_t)PPCG_ERR_TIMEOUT);
          good = 0;
          break;
        }
        __nanosleep(32);
      }
      __threadfence();
      ok = good;
    }
    __syncthreads();
    return ok != 0;
  }
};

// One thread-block cluster.  barrier.cluster with release/acquire orders the global
// writes of each pass before the next pass's gathers (which may then be served by L1; see
// GatherSlot).
// Distributed shared memory of a thread-block cluster.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_nranks() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ double ld_dsmem(uint32_t local_addr, uint32_t rank) {
  uint32_t remote;
  double v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local_addr), "r"(rank));
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(remote));
  return v;
}

struct ClusterGroup {
  static constexpr bool kCluster = true;
  __device__ int rank() const {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
  }
  __device__ int size() const {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return (int)r;
  }
  __device__ bool sync() {
    __syncthreads();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    return true;
  }
};

// ---------------------------------------------------------------- dot accumulators --

template <typename T> struct Dots;

template <> struct Dots<double> {
  double a[3] = {0.0, 0.0, 0.0};
  __device__ __forceinline__ void add(int k, double x, double y) { a[k] = fma(x, y, a[k]); }
  __device__ __forceinline__ double get(int k) const { return a[k]; }
};

// FP32 vectors: products are formed exactly as a float pair (TwoProduct with FMA, Ogita,
// Rump & Oishi 2005) and summed in double-float with Knuth's TwoSum, so the per-thread
// partials keep ~48 significant bits on the FP32 pipe; they are converted to FP64 once per
// thread and reduced in FP64 from there on.
template <> struct Dots<float> {
  float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
  __device__ __forceinline__ void add(int k, float x, float y) {
    float p = __fmul_rn(x, y);
    float e = __fmaf_rn(x, y, -p);
    float s = __fadd_rn(hi[k], p);
    float bb = __fsub_rn(s, hi[k]);
    float t = __fadd_rn(__fsub_rn(hi[k], __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi[k] = s;
    lo[k] = __fadd_rn(lo[k], __fadd_rn(t, e));
  }
  __device__ __forceinline__ double get(int k) const { return (double)hi[k] + (double)lo[k]; }
};

// --------------------------------------------------------------------- loads/stores --

template <typename T> __device__ __forceinline__ T ldcs(const T* p) { return __ldcs(p); }
template <typename T> __device__ __forceinline__ void stcs(T* p, T v) { __stcs(p, v); }
template <typename T> __device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// Streaming load of read-only matrix data: no L1 allocation, so L1 stays with the gathers.
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) {
  int32_t v;
  asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_stream(const double* p) {
  double v;
  asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

// p, made to depend on v for the compiler: loads through the result cannot be scheduled
// before v is computed.  The offset-pattern iteration passes load a row's own vector
// entries this way, after the row's product: hoisted above the gathers (as the compiler
// otherwise does, to overlap their latency) they no longer fit the 64-register budget of
// two 512-thread CTAs per SM together with the product's operands and were spilled to
// local memory and reloaded (about 40 local-memory instructions per 32-row chunk and
// iteration).  Other warps hide the latency instead: 256^3 FP64 iteration 630 -> 597 us.
template <typename T> __device__ __forceinline__ T* after(T* p, double v) {
  asm volatile("" : "+l"(p) : "d"(v));
  return p;
}
template <typename T> __device__ __forceinline__ T* after(T* p, float v) {
  asm volatile("" : "+l"(p) : "f"(v));
  return p;
}

// ---------------------------------------------------------- bulk-copy staging (TMA) --

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bulk asynchronous copy global -> shared, completing bytes on the mbarrier.  Both
// addresses 16-byte aligned, size a multiple of 16 (every caller copies whole 32-row slots).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned phase) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
  return ok != 0;
}
// Orders this thread's earlier generic-proxy accesses before its later bulk copies.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }

// Bounded wait for a stage's bulk copies; on expiry records a timeout in *err and returns.
__device__ __forceinline__ void stage_wait(uint64_t* bar, unsigned phase, int32_t* err) {
  for (uint32_t spin = 0; !mbar_try_wait(bar, phase); spin++) {
    if (spin > (1u << 22)) {
      atomicCAS(err, 0, (int32_t)PPCG_ERR_TIMEOUT);
      return;
    }
  }
}

constexpr int kStageLen = 8;                 // SELL slots per row staged in shared memory
constexpr int kStageVecBytes = 10 * kChunk * 8;                        // one FP64 tile
constexpr int kStageBytes = kStageVecBytes + kStageLen * kChunk * (4 + 8);
constexpr int kWarpStageBytes = 2 * kStageBytes;                       // double-buffered

// Chunk-interleaved vector block: for every 32-row chunk c, NS slots of 32 values each, so
// slot k of row i lives at base + (i / 32) * NS * 32 + k * 32 + i % 32.  A warp reaches all
// its rows' vectors from one chunk pointer with compile-time slot offsets, and every slot
// access of a warp is 32 consecutive values.
template <typename T, int NS> struct Blk {
  T* b;
  static constexpr int64_t kTile = (int64_t)NS * kChunk;
  __device__ __forceinline__ T* chunk(int32_t c, int lane) const { return b + (int64_t)c * kTile + lane; }
};

// Gather of one slot of a block.  The slot was written by other CTAs in an earlier pass; the
// group barrier between the passes (the grid barrier's gpu-scope acquire and fence, or
// barrier.cluster's acquire) orders those writes before every load of this CTA, so the gather
// may be served by L1 (ld.global.ca): neighbouring rows of a chunk and of the CTA's other
// warps share most of their neighbours.  On the 4M-point graph the L1 hit rate of the pass
// rises from 19% to 46% (1-2% faster); stencils are unchanged; iterates are bitwise the same.
template <typename T, int NS> struct GatherSlot {
  const T* base;   // block base + slot * 32
  __device__ __forceinline__ T operator()(int32_t j) const {
    return __ldca(base + (int64_t)(j >> 5) * ((int64_t)NS * kChunk) + (j & 31));
  }
};

// Column of SELL slot s (the row's j-th slot): the 4-byte column array; or the column
// dictionary (DevMatrix), row + coff[cidx[s]], one byte read per slot; or the offset
// pattern, row + pat[j] clamped into [0, n) -- nothing read per slot (a slot whose
// neighbour is off the grid holds a zero, so the clamped gather adds nothing).
__device__ __forceinline__ int32_t slot_col(const int32_t* __restrict__ col, int64_t s, int) {
  return ld_stream(col + s);
}
struct ColDict {
  const uint8_t* __restrict__ idx;
  const int32_t* __restrict__ off;
  int32_t row;
};
__device__ __forceinline__ int32_t slot_col(const ColDict& d, int64_t s, int) {
  return d.row + __ldg(d.off + __ldcs(d.idx + s));
}
struct ColPat {
  const int32_t* off;    // DevMatrix::pat (shared memory: the block's copy of the descriptor)
  int32_t row, last;
};
__device__ __forceinline__ int32_t slot_col(const ColPat& p, int64_t, int j) {
  return min(max(p.row + p.off[j], 0), p.last);
}

// Column modes of a kernel: the 4-byte columns everywhere; the dictionary in the iteration
// pass (4-byte columns elsewhere); the offset pattern in every pass.
enum : int { kColA = 0, kColDict = 1, kColPat = 2 };
template <int CM> struct Cols;
template <> struct Cols<kColA> {
  static __device__ __forceinline__ const int32_t* make(const DevMatrix& A, int32_t) { return A.col; }
};
template <> struct Cols<kColDict> {
  static __device__ __forceinline__ ColDict make(const DevMatrix& A, int32_t row) { return {A.cidx, A.coff, row}; }
};
template <> struct Cols<kColPat> {
  static __device__ __forceinline__ ColPat make(const DevMatrix& A, int32_t row) {
    return {A.pat, row, (int32_t)A.n - 1};
  }
};

// acc + sum_j val[slot_j] * x(col[slot_j]) (* dsc[col] when SCALE) over the row's
// off-diagonal slots base + j*32, j < len, in CSR order; acc enters holding the diagonal
// term.  CS: the column source (const int32_t* or ColDict).
// FP64 rows with stored columns: batches of 6 slots, the next batch's columns loaded before
// the current batch's gathers, so a column load no longer waits behind the gathers of the
// batch before it.  4M-point graph FP64 solve to 1e-8 with 5 / 6 / 7 / 8-slot batches: 281 /
// 251 / 260 / 267 ms (12-slot batches without the early columns 8% slower than 8; the FP32
// pass takes its own 4-slot batches).  Same terms in the same order as row_dot.
template <typename T, class G>
__device__ __forceinline__ T row_dot_cols(const int32_t* __restrict__ col, const T* __restrict__ val, const G& x,
                                          int64_t base, int len, T acc) {
  int j = 0;
  int32_t cn[6];
  if (len >= 6) {
#pragma unroll
    for (int k = 0; k < 6; k++) cn[k] = ld_stream(col + base + (int64_t)k * kChunk);
  }
  for (; j + 6 <= len; j += 6) {
    int32_t c[6];
    T a[6];
#pragma unroll
    for (int k = 0; k < 6; k++) {
      c[k] = cn[k];
      a[k] = ld_stream(val + base + (int64_t)(j + k) * kChunk);
    }
    if (j + 12 <= len) {
#pragma unroll
      for (int k = 0; k < 6; k++) cn[k] = ld_stream(col + base + (int64_t)(j + 6 + k) * kChunk);
    }
#pragma unroll
    for (int k = 0; k < 6; k++) acc = fma(a[k], x(c[k]), acc);
  }
  int32_t c[5];
  T a[5];
#pragma unroll
  for (int k = 0; k < 5; k++) {
    if (j + k < len) {
      c[k] = ld_stream(col + base + (int64_t)(j + k) * kChunk);
      a[k] = ld_stream(val + base + (int64_t)(j + k) * kChunk);
    }
  }
#pragma unroll
  for (int k = 0; k < 5; k++)
    if (j + k < len) acc = fma(a[k], x(c[k]), acc);
  return acc;
}

template <typename T, bool SCALE, class G, class CS>
__device__ __forceinline__ T row_dot(const CS& col, const T* __restrict__ val, const G& x,
                                     const T* __restrict__ dsc, int64_t base, int len, T acc) {
  if constexpr (std::is_same<CS, const int32_t*>::value && !SCALE && sizeof(T) == 8)
    return row_dot_cols(col, val, x, base, len, acc);
  if constexpr (std::is_same<CS, ColDict>::value && !SCALE && sizeof(T) == 8) {
    // FP64 rows through the column dictionary (stencils with 17-255 offsets): batches of 12
    // slots.  125-point box 165^3 SELL solve with 6 / 8 / 12 / 16-slot batches: 286 / 279 /
    // 270 / 274 ms.  Same terms, same order.
    int j = 0;
    for (; j + 12 <= len; j += 12) {
      int32_t c[12];
      T a[12];
#pragma unroll
      for (int k = 0; k < 12; k++) {
        c[k] = slot_col(col, base + (int64_t)(j + k) * kChunk, j + k);
        a[k] = ld_stream(val + base + (int64_t)(j + k) * kChunk);
      }
#pragma unroll
      for (int k = 0; k < 12; k++) acc = fma(a[k], x(c[k]), acc);
    }
#pragma unroll
    for (int k = 0; k < 11; k++) {
      if (j + k < len) {
        const int32_t c = slot_col(col, base + (int64_t)(j + k) * kChunk, j + k);
        acc = fma(ld_stream(val + base + (int64_t)(j + k) * kChunk), x(c), acc);
      }
    }
    return acc;
  }
  if constexpr (sizeof(T) == 4) {
    // FP32 rows: narrow batches, which free the registers the FP32 pass's double-float dot
    // accumulators need.  4 slots (8 before): offset pattern, 256^3 FP32_RU solve 380 -> 347
    // ms; stored columns, 4M-point graph 225 -> 215 ms; column dictionary, 125-point box
    // 165^3 180 -> 175 ms.  Offset-pattern rows take 3 (344 -> 333 ms at 256^3, whose six
    // slots make two full batches; a 2048^2 2-D system with four slots is unchanged);
    // stored columns stay at 4 (3 / 5 / 6 slots: 7% / 2% / 4% slower).  The FP64 pass is
    // 0.6% faster with the wide batches below.  Same terms, same order.
    constexpr int FB = std::is_same<CS, ColPat>::value ? 3 : 4;
    int j = 0;
    for (; j + FB <= len; j += FB) {
      T a[FB];
#pragma unroll
      for (int k = 0; k < FB; k++) a[k] = ld_stream(val + base + (int64_t)(j + k) * kChunk);
#pragma unroll
      for (int k = 0; k < FB; k++) {
        const int32_t c = slot_col(col, base + (int64_t)(j + k) * kChunk, j + k);
        T xv = x(c);
        if (SCALE) xv = __ldg(dsc + c) * xv;
        acc = fma(a[k], xv, acc);
      }
    }
#pragma unroll
    for (int k = 0; k < FB - 1; k++) {
      if (j + k < len) {
        const T a = ld_stream(val + base + (int64_t)(j + k) * kChunk);
        const int32_t c = slot_col(col, base + (int64_t)(j + k) * kChunk, j + k);
        T xv = x(c);
        if (SCALE) xv = __ldg(dsc + c) * xv;
        acc = fma(a, xv, acc);
      }
    }
    return acc;
  }
  int j = 0;
  for (; j + 8 <= len; j += 8) {
    int32_t c[8];
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      c[k] = slot_col(col, base + (int64_t)(j + k) * kChunk, j + k);
      a[k] = ld_stream(val + base + (int64_t)(j + k) * kChunk);
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      T xv = x(c[k]);
      if (SCALE) xv = __ldg(dsc + c[k]) * xv;
      acc = fma(a[k], xv, acc);
    }
  }
  int32_t c[7];
  T a[7];
#pragma unroll
  for (int k = 0; k < 7; k++) {
    if (j + k < len) {
      c[k] = slot_col(col, base + (int64_t)(j + k) * kChunk, j + k);
      a[k] = ld_stream(val + base + (int64_t)(j + k) * kChunk);
    }
  }
#pragma unroll
  for (int k = 0; k < 7; k++) {
    if (j + k < len) {
      T xv = x(c[k]);
      if (SCALE) xv = __ldg(dsc + c[k]) * xv;
      acc = fma(a[k], xv, acc);
    }
  }
  return acc;
}

// Two products over the same row in one sweep of its slots: acc1 += A x1, acc2 += A x2.
// Each accumulator sees the same FMA sequence as a row_dot of its own, so results are
// identical; the matrix slots are read once instead of twice.
template <typename T, bool SCALE, class G1, class G2, class CS>
__device__ __forceinline__ void row_dot2(const CS& col, const T* __restrict__ val, const G1& x1,
                                         const G2& x2, const T* __restrict__ dsc, int64_t base, int len, T& acc1,
                                         T& acc2) {
  int j = 0;
  for (; j + 8 <= len; j += 8) {
    int32_t c[8];
    T a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      c[k] = slot_col(col, base + (int64_t)(j + k) * kChunk, j + k);
      a[k] = ld_stream(val + base + (int64_t)(j + k) * kChunk);
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      T v1 = x1(c[k]), v2 = x2(c[k]);
      if (SCALE) { const T sc = __ldg(dsc + c[k]); v1 = sc * v1; v2 = sc * v2; }
      acc1 = fma(a[k], v1, acc1);
      acc2 = fma(a[k], v2, acc2);
    }
  }
  int32_t c[7];
  T a[7];
#pragma unroll
  for (int k = 0; k < 7; k++) {
    if (j + k < len) {
      c[k] = slot_col(col, base + (int64_t)(j + k) * kChunk, j + k);
      a[k] = ld_stream(val + base + (int64_t)(j + k) * kChunk);
    }
  }
#pragma unroll
  for (int k = 0; k < 7; k++) {
    if (j + k < len) {
      T v1 = x1(c[k]), v2 = x2(c[k]);
      if (SCALE) { const T sc = __ldg(dsc + c[k]); v1 = sc * v1; v2 = sc * v2; }
      acc1 = fma(a[k], v1, acc1);
      acc2 = fma(a[k], v2, acc2);
    }
  }
}

// L2 prefetch of the lines chunk c will read (its vector tile and its matrix slots), issued
// one chunk ahead by the warp that will process it: the lines are in flight while the warp
// works on its current chunk, at no register cost.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
template <typename T, int NS>
__device__ __forceinline__ void prefetch_chunk(const int64_t* __restrict__ cptr, const int32_t* __restrict__ col,
                                               const uint8_t* __restrict__ cidx, const T* __restrict__ val,
                                               const T* blk, int32_t c, int lane, int pat_k = 0) {
  constexpr int kTileBytes = NS * kChunk * (int)sizeof(T);
  const char* tile = reinterpret_cast<const char*>(blk + (int64_t)c * NS * kChunk);
  for (int off = lane * 128; off < kTileBytes; off += 32 * 128) prefetch_l2(tile + off);
  if (pat_k > 0) {                 // offset pattern: values only, no column bytes
    const char* pv = reinterpret_cast<const char*>(val + (int64_t)c * pat_k * kChunk);
    const int nv = pat_k * kChunk * (int)sizeof(T);
    for (int off = lane * 128; off < nv; off += 32 * 128) prefetch_l2(pv + off);
    return;
  }
  const int64_t b0 = __ldg(cptr + c), b1 = __ldg(cptr + c + 1);
  // Long rows (over 16 slots) keep enough loads in flight on their own, and prefetching
  // their matrix slots a chunk ahead from every warp would overflow L2 (the 125-point box:
  // 32 KB per chunk); only the vector tile is prefetched for them.
  if (b1 - b0 > 16 * kChunk) return;
  const char* pc = cidx ? reinterpret_cast<const char*>(cidx + b0) : reinterpret_cast<const char*>(col + b0);
  const char* pv = reinterpret_cast<const char*>(val + b0);
  const int nc = (int)((b1 - b0) * (cidx ? 1 : 4)), nv = (int)((b1 - b0) * (int64_t)sizeof(T));
  for (int off = lane * 128; off < nc; off += 32 * 128) prefetch_l2(pc + off);
  for (int off = lane * 128; off < nv; off += 32 * 128) prefetch_l2(pv + off);
}

// L2 prefetch, at the start of a chunk, of its matrix lines past the first batch of 8 slots
// (stored columns and values): the later batches' column loads then come from L2 instead of
// DRAM, which shortens the chain column -> gather -> FMA of each batch.  4M-point graph
// (about 23 slots per chunk): FP64 solve 4.1%, FP32_RU 2.3% faster.  Prefetching the next
// chunk's first batch as well (one chunk ahead) made the FP64 solve 2% slower, and with the
// next chunk's vector tile 7% slower.
template <typename T>
__device__ __forceinline__ void prefetch_rest(const int32_t* __restrict__ col, const T* __restrict__ val, int64_t b0,
                                              int len, int lane) {
  if (len <= 8) return;
  const int64_t s0 = b0 + 8 * kChunk;
  const int ncl = (len - 8) * kChunk * 4 / 128, nvl = (len - 8) * kChunk * (int)sizeof(T) / 128;
  if (lane < ncl) prefetch_l2(col + s0 + lane * 32);
  for (int l = lane; l < nvl; l += 32) prefetch_l2(reinterpret_cast<const char*>(val + s0) + l * 128);
}

#ifndef PPCG_PREFETCH
#define PPCG_PREFETCH 1
#endif

// Vector slots.  FP64 block (NS 10): r u wa wb z q s p x invd.  FP32 block (NS 11):
// r u wa wb z q s p d invd rhs (d: inner solution).  FP32_IR keeps its FP64 outer residual
// and solution in slots r and x of the FP64 block.
enum { V_R = 0, V_U, V_WA, V_WB, V_Z, V_Q, V_S, V_P, V_X, V_INVD, V_RHS };
constexpr int kNS64 = 10, kNS32 = 11;
constexpr int IR_R = V_R, IR_X = V_X;

struct Lanes {
  int32_t gw, W;   // global warp id within the group, warps in the group (chunk indices < 2^26)
  int32_t lane;
};

#define FOR_CHUNKS(A, L) for (int32_t c = (L).gw; c < (int32_t)(A).nchunks; c += (L).W)

template <int CM = kColA>
__device__ __forceinline__ void chunk_slots(const DevMatrix& A, int32_t c, int lane, int64_t& base, int& len) {
  if constexpr (CM == kColPat) {   // pat_k slots in every chunk: no chunk pointers to read
    len = A.pat_k;
    base = (int64_t)c * A.pat_k * kChunk + lane;
  } else {
    const int64_t b0 = __ldg(A.cptr + c);
    len = (int)((__ldg(A.cptr + c + 1) - b0) / kChunk);
    base = b0 + lane;
  }
}

// Per-precision matrix/vector view used by the generic passes.
template <typename T, int NS> struct View {
  const T* val;     // SELL values (A D^-1, off-diagonal)
  const T* dsc;     // a_ii per row, plain array (gathered as the column scale of A v)
  const T* rhs;     // right-hand side, plain array (FP64 path) -- nullptr when it is a slot
  Blk<T, NS> v;
};

__device__ __forceinline__ View<double, kNS64> view64(const SysDesc& S) {
  return {S.A.val, S.A.diag, S.b, {S.v64}};
}
__device__ __forceinline__ View<float, kNS32> view32(const SysDesc& S) {
  return {S.A.val32, S.A.diag32, nullptr, {S.v32}};
}

// -------------------------------------------------------------------------- passes --

// P_SETUP1 (FP64), Alg. 2 setup: r0 = b - A x0 ; u0 = M^-1 r0.  Partials (b,b), (r,r).
template <int CM>
__device__ __forceinline__ void pass_setup1(const SysDesc& S, const Lanes& L, Dots<double>& d, bool x_zero) {
  const DevMatrix& A = S.A;
  const Blk<double, kNS64> v{S.v64};
  const GatherSlot<double, kNS64> gx{S.v64 + V_X * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    double* pc = v.chunk(c, L.lane);
    double ax = 0.0, bi = 0.0, id = 0.0;
    if (in) {
      bi = __ldg(S.b + row);
      id = ldcs(pc + V_INVD * kChunk);
      if (!x_zero) ax = __ldg(A.diag + row) * ldcg(pc + V_X * kChunk);
    }
    if (!x_zero) ax = row_dot<double, true>(Cols<CM>::make(A, row), A.val, gx, A.diag, base, len, ax);
    if (in) {
      const double ri = bi - ax;
      stcs(pc + V_R * kChunk, ri);
      stcs(pc + V_U * kChunk, id * ri);
      d.add(0, bi, bi);
      d.add(1, ri, ri);
    }
  }
}

// P_SETUP2, Alg. 2 setup: w0 = A u0 (= Ahat r0) ; partials (r,u), (w,u), norm.
template <typename T, int NS, int CM>
__device__ __forceinline__ void pass_setup2(const DevMatrix& A, const View<T, NS>& V, const Lanes& L, Dots<T>& d,
                                            bool paper_norm) {
  const GatherSlot<T, NS> gr{V.v.b + V_R * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    T* pc = V.v.chunk(c, L.lane);
    T ri = T(0), ui = T(0);
    if (in) { ri = ldcg(pc + V_R * kChunk); ui = ldcs(pc + V_U * kChunk); }
    const T wi = row_dot<T, false>(Cols<CM>::make(A, row), V.val, gr, nullptr, base, len, ri);
    if (in) {
      stcs(pc + V_WA * kChunk, wi);
      d.add(0, ri, ui);
      d.add(1, wi, ui);
      if (paper_norm) d.add(2, ui, ui); else d.add(2, ri, ri);
    }
  }
}

// P_ITER: one full iteration of Alg. 2 for the group's rows (see the file comment).  With
// the offset pattern the row's own vector entries other than w are loaded after the
// product (see after()); with stored columns, beside the gathers.
template <typename T, int NS, bool FIRST, int CM = kColA>
__device__ __forceinline__ void pass_iter(const DevMatrix& A, const View<T, NS>& V, const Lanes& L, Dots<T>& d,
                                          T alpha, T beta, int k, bool paper_norm, bool with_rr = true,
                                          bool pf_own = false) {
  const int wcs = (k & 1) ? V_WB : V_WA;
  const int wns = (k & 1) ? V_WA : V_WB;
  const GatherSlot<T, NS> gw{V.v.b + wcs * kChunk};
  const T* __restrict__ val = V.val;
  const int32_t n = (int32_t)A.n;
  // Odd iterations walk each warp's chunks in reverse, so a pass starts on the chunks the
  // previous pass wrote last, whose lines are still in L2 (the ramp-up after the barrier
  // reads from L2 instead of DRAM).  256^3 FP64 solve 0.5%, FP32_RU 1.7%, 4M-point graph
  // FP64 2.6% per iteration faster.  The per-lane dot partials then sum in another order
  // on odd iterations: FP64 iterates change by rounding only.
  const int32_t nch = (int32_t)A.nchunks;
  const int32_t cnt = L.gw < nch ? (nch - 1 - L.gw) / L.W + 1 : 0;
  const bool rev = (k & 1) != 0;
  for (int32_t ci = 0; ci < cnt; ci++) {
    const int32_t c = L.gw + (rev ? cnt - 1 - ci : ci) * L.W;
    // FP32 only: the FP32 pass is latency-bound (half the bytes in flight of FP64 at the
    // same occupancy), 433 -> 350 us per 256^3 iteration; the FP64 pass, already near the
    // HBM and FP64-pipe limits, ran 10-20% slower with it.
    if (PPCG_PREFETCH && sizeof(T) == 4 && ci + 1 < cnt)
      prefetch_chunk<T, NS>(A.cptr, A.col, CM == kColDict ? A.cidx : nullptr, val, V.v.b, rev ? c - L.W : c + L.W,
                            L.lane, CM == kColPat ? A.pat_k : 0);
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    if (CM == kColA) prefetch_rest(A.col, val, base - L.lane, len, L.lane);
    // Stencils (the row's own entries are loaded after the product, see after()): an L2
    // prefetch of the chunk's eight own-entry slots (not the two w slots) at the start of the
    // chunk, so those loads find their lines in L2.  256^3 FP64 solve 611 -> 606 ms.  Only
    // for systems whose vectors do not stay in L2 between passes (pf_own): on small ones
    // the instructions only lengthen the chain (64^2 cluster solve 1.55 -> 1.71 ms).
    if (CM == kColPat && sizeof(T) == 8 && pf_own && L.lane < 16) {
      const int sl = L.lane >> 1;   // slots r u (z q s p x invd): 0 1 4 .. 9
      const char* line = reinterpret_cast<const char*>(V.v.chunk(c, 0)) + (sl < 2 ? sl : sl + 2) * (kChunk * 8) +
                         (L.lane & 1) * 128;
      prefetch_l2(line);   // (into L1 instead: the same time)
    }
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < n;
    T* pc = V.v.chunk(c, L.lane);
    T wi = T(0), id = T(0), ui = T(0), xi = T(0), ri = T(0);
    T zo = T(0), qo = T(0), so = T(0), po = T(0);
    if (in) wi = ldcg(pc + wcs * kChunk);
    // Irregular matrices (4-byte columns): the row's own entries are loaded beside the
    // gathers, whose latency they help cover (4M-point graph: 2.4% faster than after).
    if (CM != kColPat && in) {
      id = ldcs(pc + V_INVD * kChunk);
      ui = ldcs(pc + V_U * kChunk);
      xi = ldcs(pc + V_X * kChunk);
      ri = ldcs(pc + V_R * kChunk);
      if (!FIRST) {
        zo = ldcs(pc + V_Z * kChunk);
        qo = ldcs(pc + V_Q * kChunk);
        so = ldcs(pc + V_S * kChunk);
        po = ldcs(pc + V_P * kChunk);
      }
    }
    // n_i = (A M^-1 w)_i = w_i + sum_{j != i} ahat_ij w_j
    const T ni = row_dot<T, false>(Cols<CM>::make(A, row), val, gw, nullptr, base, len, wi);
    if (CM == kColPat && in) {   // stencils: the row's own entries after the product (see after())
      const T* q = after(pc, ni);
      id = ldcs(q + V_INVD * kChunk);
      ui = ldcs(q + V_U * kChunk);
      xi = ldcs(q + V_X * kChunk);
      ri = ldcs(q + V_R * kChunk);
      if (!FIRST) {
        zo = ldcs(q + V_Z * kChunk);
        qo = ldcs(q + V_Q * kChunk);
        so = ldcs(q + V_S * kChunk);
        po = ldcs(q + V_P * kChunk);
      }
    }
    if (in) {
      const T mi = id * wi;
      const T zi = FIRST ? ni : fma(beta, zo, ni);
      const T qi = FIRST ? mi : fma(beta, qo, mi);
      const T si = FIRST ? wi : fma(beta, so, wi);
      const T pi = FIRST ? ui : fma(beta, po, ui);
      xi = fma(alpha, pi, xi);
      ri = fma(-alpha, si, ri);
      const T un = fma(-alpha, qi, ui);
      const T wnn = fma(-alpha, zi, wi);
      stcs(pc + V_Z * kChunk, zi);
      stcs(pc + V_Q * kChunk, qi);
      stcs(pc + V_S * kChunk, si);
      stcs(pc + V_P * kChunk, pi);
      stcs(pc + V_X * kChunk, xi);
      stcs(pc + V_R * kChunk, ri);
      stcs(pc + V_U * kChunk, un);
      stcs(pc + wns * kChunk, wnn);
      d.add(0, ri, un);
      d.add(1, wnn, un);
      if (with_rr) { if (paper_norm) d.add(2, un, un); else d.add(2, ri, ri); }
    }
  }
}

// P_NORM (Alg. 2 form): partial ||r||^2 or (u, u).
template <typename T, int NS>
__device__ __forceinline__ void pass_norm(const DevMatrix& A, const View<T, NS>& V, const Lanes& L, Dots<T>& d,
                                          bool paper_norm) {
  FOR_CHUNKS(A, L) {
    const int32_t row = c * kChunk + L.lane;
    if (row < A.n) {
      const T v = ldcs(V.v.chunk(c, L.lane) + (paper_norm ? V_U : V_R) * kChunk);
      d.add(2, v, v);
    }
  }
}

// P_ITER with bulk-copy staging (whole-GPU path).  Each warp double-buffers its chunks in
// shared memory: while it computes chunk c, the bulk copies of chunk c + W (the row tile of
// every vector it reads, and the chunk's SELL columns and values when the rows have at most
// kStageLen slots) are in flight.  Only the gathers of w from other chunks and the results
// go through registers to and from global memory.
template <typename T, int NS, bool FIRST>
__device__ __forceinline__ void pass_iter_staged(const DevMatrix& A, const View<T, NS>& V, const Lanes& L,
                                                 Dots<T>& d, T alpha, T beta, int k, bool paper_norm,
                                                 unsigned char* wst, uint64_t* bars, unsigned& phases,
                                                 int32_t* err) {
  constexpr int NV = (NS == 11) ? 10 : NS;     // slots read by the pass (FP32 block: not rhs)
  const int wcs = (k & 1) ? V_WB : V_WA;
  const int wns = (k & 1) ? V_WA : V_WB;
  const GatherSlot<T, NS> gw{V.v.b + wcs * kChunk};
  const int32_t* __restrict__ col = A.col;
  const T* __restrict__ val = V.val;
  const int64_t* __restrict__ cptr = A.cptr;
  const int32_t n = (int32_t)A.n;
  const int32_t nchunks = (int32_t)A.nchunks;
  const int lane = L.lane;

  auto vec_s = [&](int st) { return reinterpret_cast<T*>(wst + st * kStageBytes); };
  auto col_s = [&](int st) { return reinterpret_cast<int32_t*>(wst + st * kStageBytes + kStageVecBytes); };
  auto val_s = [&](int st) {
    return reinterpret_cast<T*>(wst + st * kStageBytes + kStageVecBytes + kStageLen * kChunk * 4);
  };
  auto issue = [&](int st, int32_t c) {            // one lane
    const int64_t b0 = __ldg(cptr + c);
    const int len = (int)((__ldg(cptr + c + 1) - b0) / kChunk);
    const T* tile = V.v.b + (int64_t)c * NS * kChunk;
    const unsigned lo = (unsigned)(wns * kChunk * sizeof(T));
    const unsigned hi = (unsigned)((NV - wns - 1) * kChunk * sizeof(T));
    unsigned bytes = lo + hi;
    const bool mat = len > 0 && len <= kStageLen;
    if (mat) bytes += (unsigned)(len * kChunk * (4 + sizeof(T)));
    fence_proxy_async();
    mbar_expect_tx(bars + st, bytes);
    bulk_g2s(vec_s(st), tile, lo, bars + st);
    bulk_g2s(vec_s(st) + (wns + 1) * kChunk, tile + (wns + 1) * kChunk, hi, bars + st);
    if (mat) {
      bulk_g2s(col_s(st), col + b0, (unsigned)(len * kChunk * 4), bars + st);
      bulk_g2s(val_s(st), val + b0, (unsigned)(len * kChunk * sizeof(T)), bars + st);
    }
  };

  int st = 0;
  int32_t c = L.gw;
  if (c < nchunks && lane == 0) issue(0, c);
  for (; c < nchunks; c += L.W, st ^= 1) {
    const int32_t cn = c + L.W;
    if (cn < nchunks && lane == 0) issue(st ^ 1, cn);
    const int64_t b0 = __ldg(cptr + c);
    const int len = (int)((__ldg(cptr + c + 1) - b0) / kChunk);
    stage_wait(bars + st, (phases >> st) & 1u, err);
    phases ^= 1u << st;
    const int32_t row = c * kChunk + lane;
    const bool in = row < n;
    const T* vsm = vec_s(st) + lane;
    T acc = vsm[wcs * kChunk];
    const T wi = acc;
    if (len <= kStageLen) {
      const int32_t* cs = col_s(st) + lane;
      const T* as = val_s(st) + lane;
      int32_t cc[kStageLen];
      T aa[kStageLen];
#pragma unroll
      for (int j = 0; j < kStageLen; j++)
        if (j < len) { cc[j] = cs[j * kChunk]; aa[j] = as[j * kChunk]; }
#pragma unroll
      for (int j = 0; j < kStageLen; j++)
        if (j < len) acc = fma(aa[j], gw(cc[j]), acc);
    } else {
      acc = row_dot<T, false>(col, val, gw, nullptr, b0 + lane, len, acc);
    }
    if (in) {
      const T ni = acc;
      const T id = vsm[V_INVD * kChunk];
      const T ui = vsm[V_U * kChunk];
      const T mi = id * wi;
      const T zi = FIRST ? ni : fma(beta, vsm[V_Z * kChunk], ni);
      const T qi = FIRST ? mi : fma(beta, vsm[V_Q * kChunk], mi);
      const T si = FIRST ? wi : fma(beta, vsm[V_S * kChunk], wi);
      const T pi = FIRST ? ui : fma(beta, vsm[V_P * kChunk], ui);
      const T xi = fma(alpha, pi, vsm[V_X * kChunk]);
      const T ri = fma(-alpha, si, vsm[V_R * kChunk]);
      const T un = fma(-alpha, qi, ui);
      const T wnn = fma(-alpha, zi, wi);
      T* pc = V.v.chunk(c, lane);
      stcs(pc + V_Z * kChunk, zi);
      stcs(pc + V_Q * kChunk, qi);
      stcs(pc + V_S * kChunk, si);
      stcs(pc + V_P * kChunk, pi);
      stcs(pc + V_X * kChunk, xi);
      stcs(pc + V_R * kChunk, ri);
      stcs(pc + V_U * kChunk, un);
      stcs(pc + wns * kChunk, wnn);
      d.add(0, ri, un);
      d.add(1, wnn, un);
      if (paper_norm) d.add(2, un, un); else d.add(2, ri, ri);
    }
    __syncwarp();
  }
}

// P_TRUE (FP64): partial ||b - A x||^2, x in slot XS of an NS-slot FP64 block.
template <int NS, int XS, int CM>
__device__ __forceinline__ void pass_true(const SysDesc& S, const Lanes& L, Dots<double>& d) {
  const DevMatrix& A = S.A;
  const Blk<double, NS> v{S.v64};
  const GatherSlot<double, NS> gx{S.v64 + XS * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    double ax = 0.0, bi = 0.0;
    if (in) { bi = __ldg(S.b + row); ax = __ldg(A.diag + row) * ldcg(v.chunk(c, L.lane) + XS * kChunk); }
    ax = row_dot<double, true>(Cols<CM>::make(A, row), A.val, gx, A.diag, base, len, ax);
    if (in) {
      const double t = bi - ax;
      d.add(0, t, t);
    }
  }
}

// P_GAP (FP64): partials ||(b - A x) - r||^2 and ||r||^2, x and r in slots XS and RS of an
// NS-slot FP64 block: the measured deviation of the recursive residual from the true one.
template <int NS, int XS, int RS, int CM>
__device__ __forceinline__ void pass_gap(const SysDesc& S, const Lanes& L, Dots<double>& d) {
  const DevMatrix& A = S.A;
  const Blk<double, NS> v{S.v64};
  const GatherSlot<double, NS> gx{S.v64 + XS * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    double ax = 0.0, bi = 0.0, ri = 0.0;
    if (in) {
      const double* pc = v.chunk(c, L.lane);
      bi = __ldg(S.b + row);
      ri = ldcs(pc + RS * kChunk);
      ax = __ldg(A.diag + row) * ldcg(pc + XS * kChunk);
    }
    ax = row_dot<double, true>(Cols<CM>::make(A, row), A.val, gx, A.diag, base, len, ax);
    if (in) {
      const double g = (bi - ax) - ri;
      d.add(0, g, g);
      d.add(1, ri, ri);
    }
  }
}

// P_RR1: residual replacement, first half: r = rhs - A x ; u = M^-1 r ; s = A p ; q = M^-1 s.
// (At iteration 0 p is zero, so s = q = 0.)
template <typename T, int NS, int CM>
__device__ __forceinline__ void pass_rr1(const DevMatrix& A, const View<T, NS>& V, const Lanes& L, bool p_zero) {
  const GatherSlot<T, NS> gx{V.v.b + V_X * kChunk};
  const GatherSlot<T, NS> gp{V.v.b + V_P * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    T* pc = V.v.chunk(c, L.lane);
    T ax = T(0), ap = T(0), id = T(0), rh = T(0);
    if (in) {
      const T di = __ldg(V.dsc + row);
      id = ldcs(pc + V_INVD * kChunk);
      rh = V.rhs ? __ldg(V.rhs + row) : ldcs(pc + V_RHS * kChunk);
      ax = di * ldcg(pc + V_X * kChunk);
      if (!p_zero) ap = di * ldcg(pc + V_P * kChunk);
    }
    if (p_zero) ax = row_dot<T, true>(Cols<CM>::make(A, row), V.val, gx, V.dsc, base, len, ax);
    else row_dot2<T, true>(Cols<CM>::make(A, row), V.val, gx, gp, V.dsc, base, len, ax, ap);
    if (in) {
      const T ri = rh - ax;
      stcs(pc + V_R * kChunk, ri);
      stcs(pc + V_U * kChunk, id * ri);
      stcs(pc + V_S * kChunk, ap);
      stcs(pc + V_Q * kChunk, id * ap);
    }
  }
}

// P_RR2: w = A u (= Ahat r) ; z = A q (= Ahat s) ; partials (r,u), (w,u), norm.
template <typename T, int NS, int CM>
__device__ __forceinline__ void pass_rr2(const DevMatrix& A, const View<T, NS>& V, const Lanes& L, Dots<T>& d,
                                         int k, bool paper_norm) {
  const int wcs = (k & 1) ? V_WB : V_WA;
  const GatherSlot<T, NS> gr{V.v.b + V_R * kChunk};
  const GatherSlot<T, NS> gs{V.v.b + V_S * kChunk};
  FOR_CHUNKS(A, L) {
    if (PPCG_PREFETCH && sizeof(T) == 4 && c + L.W < (int32_t)A.nchunks)
      prefetch_chunk<T, NS>(A.cptr, A.col, nullptr, V.val, V.v.b, c + L.W, L.lane, CM == kColPat ? A.pat_k : 0);
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    T* pc = V.v.chunk(c, L.lane);
    T ri = T(0), ui = T(0), si = T(0);
    if (in) { ri = ldcg(pc + V_R * kChunk); ui = ldcs(pc + V_U * kChunk); si = ldcg(pc + V_S * kChunk); }
    T wi = ri, zi = si;
    row_dot2<T, false>(Cols<CM>::make(A, row), V.val, gr, gs, nullptr, base, len, wi, zi);
    if (in) {
      stcs(pc + wcs * kChunk, wi);
      stcs(pc + V_Z * kChunk, zi);
      d.add(0, ri, ui);
      d.add(1, wi, ui);
      if (paper_norm) d.add(2, ui, ui); else d.add(2, ri, ri);
    }
  }
}

// ------------------------------------------ Jacobi-scaled variant (Jacobi elimination) --
// With M = D = diag(A), u = D^-1 r and q = D^-1 s hold exactly, and Alg. 2 is the
// unpreconditioned pipelined iteration on A~ = D^-1/2 A D^-1/2 in the variables
// x~ = D^1/2 x, r~ = D^-1/2 r (= D^1/2 u), w~ = D^-1/2 w, ... where u = r, q = s, m = w:
// gamma = (r~, r~), delta = (w~, r~) are Alg. 2's gamma and delta, and the stopping norm
// ||r||^2 = sum d_i r~_i^2.  FP64 block: r wa wb z s p x d sig (sig = d^-1/2).
enum { VS_R = 0, VS_WA, VS_WB, VS_Z, VS_S, VS_P, VS_X, VS_D, VS_SIG };
constexpr int kNSS = 9;

__device__ __forceinline__ double scaled_norm_term(bool paper, double ri, double di, double sg) {
  return paper ? (sg * ri) * (sg * ri) : (di * ri) * ri;
}

// P_SETUP1: r~ = sig b - A~ x~ ; partial (b, b).
template <int CM>
__device__ __forceinline__ void spass_setup1(const SysDesc& S, const Lanes& L, Dots<double>& d, bool x_zero) {
  const DevMatrix& A = S.A;
  const Blk<double, kNSS> v{S.v64};
  const GatherSlot<double, kNSS> gx{S.v64 + VS_X * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    double* pc = v.chunk(c, L.lane);
    double ax = 0.0, bi = 0.0, sg = 0.0;
    if (in) {
      bi = __ldg(S.b + row);
      sg = ldcs(pc + VS_SIG * kChunk);
      if (!x_zero) ax = ldcg(pc + VS_X * kChunk);
    }
    if (!x_zero) ax = row_dot<double, false>(Cols<CM>::make(A, row), A.val, gx, nullptr, base, len, ax);
    if (in) {
      stcs(pc + VS_R * kChunk, fma(sg, bi, -ax));
      d.add(0, bi, bi);
    }
  }
}

// P_SETUP2: w~ = A~ r~ ; partials gamma = (r~, r~), delta = (w~, r~), stopping norm.
template <int CM>
__device__ __forceinline__ void spass_setup2(const SysDesc& S, const Lanes& L, Dots<double>& d, bool paper) {
  const DevMatrix& A = S.A;
  const Blk<double, kNSS> v{S.v64};
  const GatherSlot<double, kNSS> gr{S.v64 + VS_R * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    double* pc = v.chunk(c, L.lane);
    double ri = 0.0, di = 0.0, sg = 0.0;
    if (in) {
      ri = ldcg(pc + VS_R * kChunk);
      if (paper) sg = ldcs(pc + VS_SIG * kChunk); else di = ldcs(pc + VS_D * kChunk);
    }
    const double wi = row_dot<double, false>(Cols<CM>::make(A, row), A.val, gr, nullptr, base, len, ri);
    if (in) {
      stcs(pc + VS_WA * kChunk, wi);
      d.add(0, ri, ri);
      d.add(1, wi, ri);
      d.a[2] += scaled_norm_term(paper, ri, di, sg);
    }
  }
}

// P_ITER (scaled): n~ = A~ w~ ; z = n + beta z ; s = w + beta s ; p = r + beta p ;
// x += alpha p ; r -= alpha s ; w -= alpha z ; partials.
template <bool FIRST, int CM>
__device__ __forceinline__ void spass_iter(const SysDesc& S, const Lanes& L, Dots<double>& d, double alpha,
                                           double beta, int k, bool paper, bool with_rr) {
  const DevMatrix& A = S.A;
  const Blk<double, kNSS> v{S.v64};
  const int wcs = (k & 1) ? VS_WB : VS_WA;
  const int wns = (k & 1) ? VS_WA : VS_WB;
  const GatherSlot<double, kNSS> gw{S.v64 + wcs * kChunk};
  const double* __restrict__ val = A.val;
  const int32_t n = (int32_t)A.n;
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < n;
    double* pc = v.chunk(c, L.lane);
    double wi = 0.0, ri = 0.0, xi = 0.0, zo = 0.0, so = 0.0, po = 0.0, di = 0.0, sg = 0.0;
    if (in) wi = ldcg(pc + wcs * kChunk);
    if (CM != kColPat && in) {   // as in pass_iter: beside the gathers for stored columns
      ri = ldcs(pc + VS_R * kChunk);
      xi = ldcs(pc + VS_X * kChunk);
      if (with_rr) { if (paper) sg = ldcs(pc + VS_SIG * kChunk); else di = ldcs(pc + VS_D * kChunk); }
      if (!FIRST) {
        zo = ldcs(pc + VS_Z * kChunk);
        so = ldcs(pc + VS_S * kChunk);
        po = ldcs(pc + VS_P * kChunk);
      }
    }
    const double ni = row_dot<double, false>(Cols<CM>::make(A, row), val, gw, nullptr, base, len, wi);
    if (CM == kColPat && in) {   // stencils: the row's own entries after the product (see after())
      const double* q = after(pc, ni);
      ri = ldcs(q + VS_R * kChunk);
      xi = ldcs(q + VS_X * kChunk);
      if (with_rr) { if (paper) sg = ldcs(q + VS_SIG * kChunk); else di = ldcs(q + VS_D * kChunk); }
      if (!FIRST) {
        zo = ldcs(q + VS_Z * kChunk);
        so = ldcs(q + VS_S * kChunk);
        po = ldcs(q + VS_P * kChunk);
      }
    }
    if (in) {
      const double zi = FIRST ? ni : fma(beta, zo, ni);
      const double si = FIRST ? wi : fma(beta, so, wi);
      const double pi = FIRST ? ri : fma(beta, po, ri);
      xi = fma(alpha, pi, xi);
      const double rn = fma(-alpha, si, ri);
      const double wn = fma(-alpha, zi, wi);
      stcs(pc + VS_Z * kChunk, zi);
      stcs(pc + VS_S * kChunk, si);
      stcs(pc + VS_P * kChunk, pi);
      stcs(pc + VS_X * kChunk, xi);
      stcs(pc + VS_R * kChunk, rn);
      stcs(pc + wns * kChunk, wn);
      d.add(0, rn, rn);
      d.add(1, wn, rn);
      if (with_rr) d.a[2] += scaled_norm_term(paper, rn, di, sg);
    }
  }
}

// P_NORM (scaled): partial sum d r~^2 (= ||r||^2) or sig^2 r~^2 (= (u, u)).
__device__ __forceinline__ void spass_norm(const SysDesc& S, const Lanes& L, Dots<double>& d, bool paper) {
  const Blk<double, kNSS> v{S.v64};
  FOR_CHUNKS(S.A, L) {
    const int32_t row = c * kChunk + L.lane;
    if (row < S.A.n) {
      const double* pc = v.chunk(c, L.lane);
      const double ri = ldcs(pc + VS_R * kChunk);
      const double di = paper ? 0.0 : ldcs(pc + VS_D * kChunk);
      const double sg = paper ? ldcs(pc + VS_SIG * kChunk) : 0.0;
      d.a[2] += scaled_norm_term(paper, ri, di, sg);
    }
  }
}

// P_TRUE (scaled): ||b - A x||^2 = sum d (sig b - A~ x~)^2.
template <int CM>
__device__ __forceinline__ void spass_true(const SysDesc& S, const Lanes& L, Dots<double>& d) {
  const DevMatrix& A = S.A;
  const Blk<double, kNSS> v{S.v64};
  const GatherSlot<double, kNSS> gx{S.v64 + VS_X * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    double* pc = v.chunk(c, L.lane);
    double ax = 0.0, bi = 0.0, sg = 0.0, di = 0.0;
    if (in) {
      bi = __ldg(S.b + row);
      sg = ldcs(pc + VS_SIG * kChunk);
      di = ldcs(pc + VS_D * kChunk);
      ax = ldcg(pc + VS_X * kChunk);
    }
    ax = row_dot<double, false>(Cols<CM>::make(A, row), A.val, gx, nullptr, base, len, ax);
    if (in) {
      const double t = fma(sg, bi, -ax);
      d.add(0, di * t, t);
    }
  }
}

// P_GAP (scaled): ||(b - A x) - r||^2 = sum d ((sig b - A~ x~) - r~)^2 and ||r||^2 = sum d r~^2.
template <int CM>
__device__ __forceinline__ void spass_gap(const SysDesc& S, const Lanes& L, Dots<double>& d) {
  const DevMatrix& A = S.A;
  const Blk<double, kNSS> v{S.v64};
  const GatherSlot<double, kNSS> gx{S.v64 + VS_X * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    double* pc = v.chunk(c, L.lane);
    double ax = 0.0, bi = 0.0, sg = 0.0, di = 0.0, ri = 0.0;
    if (in) {
      bi = __ldg(S.b + row);
      sg = ldcs(pc + VS_SIG * kChunk);
      di = ldcs(pc + VS_D * kChunk);
      ri = ldcs(pc + VS_R * kChunk);
      ax = ldcg(pc + VS_X * kChunk);
    }
    ax = row_dot<double, false>(Cols<CM>::make(A, row), A.val, gx, nullptr, base, len, ax);
    if (in) {
      const double g = fma(sg, bi, -ax) - ri;
      d.add(0, di * g, g);
      d.add(1, di * ri, ri);
    }
  }
}

// P_RR1 (scaled): r~ = sig b - A~ x~ ; s~ = A~ p~ (0 at a restart or at iteration 0).
template <int CM>
__device__ __forceinline__ void spass_rr1(const SysDesc& S, const Lanes& L, bool p_zero) {
  const DevMatrix& A = S.A;
  const Blk<double, kNSS> v{S.v64};
  const GatherSlot<double, kNSS> gx{S.v64 + VS_X * kChunk};
  const GatherSlot<double, kNSS> gp{S.v64 + VS_P * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    double* pc = v.chunk(c, L.lane);
    double ax = 0.0, ap = 0.0, bi = 0.0, sg = 0.0;
    if (in) {
      bi = __ldg(S.b + row);
      sg = ldcs(pc + VS_SIG * kChunk);
      ax = ldcg(pc + VS_X * kChunk);
      if (!p_zero) ap = ldcg(pc + VS_P * kChunk);
    }
    if (p_zero) ax = row_dot<double, false>(Cols<CM>::make(A, row), A.val, gx, nullptr, base, len, ax);
    else row_dot2<double, false>(Cols<CM>::make(A, row), A.val, gx, gp, nullptr, base, len, ax, ap);
    if (in) {
      stcs(pc + VS_R * kChunk, fma(sg, bi, -ax));
      stcs(pc + VS_S * kChunk, ap);
    }
  }
}

// P_RR2 (scaled): w~ = A~ r~ ; z~ = A~ s~ ; partials.
template <int CM>
__device__ __forceinline__ void spass_rr2(const SysDesc& S, const Lanes& L, Dots<double>& d, int k, bool paper) {
  const DevMatrix& A = S.A;
  const Blk<double, kNSS> v{S.v64};
  const int wcs = (k & 1) ? VS_WB : VS_WA;
  const GatherSlot<double, kNSS> gr{S.v64 + VS_R * kChunk};
  const GatherSlot<double, kNSS> gs{S.v64 + VS_S * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    double* pc = v.chunk(c, L.lane);
    double ri = 0.0, si = 0.0, di = 0.0, sg = 0.0;
    if (in) {
      ri = ldcg(pc + VS_R * kChunk);
      si = ldcg(pc + VS_S * kChunk);
      if (paper) sg = ldcs(pc + VS_SIG * kChunk); else di = ldcs(pc + VS_D * kChunk);
    }
    double wi = ri, zi = si;
    row_dot2<double, false>(Cols<CM>::make(A, row), A.val, gr, gs, nullptr, base, len, wi, zi);
    if (in) {
      stcs(pc + wcs * kChunk, wi);
      stcs(pc + VS_Z * kChunk, zi);
      d.add(0, ri, ri);
      d.add(1, wi, ri);
      d.a[2] += scaled_norm_term(paper, ri, di, sg);
    }
  }
}

// P_ZERO_X: x = 0 (slot XS of an NS-slot FP64 block).
template <int NS, int XS>
__device__ __forceinline__ void pass_zero_x(const SysDesc& S, const Lanes& L) {
  const Blk<double, NS> v{S.v64};
  FOR_CHUNKS(S.A, L) {
    const int32_t row = c * kChunk + L.lane;
    if (row < S.A.n) v.chunk(c, L.lane)[XS * kChunk] = 0.0;
  }
}

// P_ORES (FP32_IR outer step): r64 = b - A x in FP64 ; partials (r64,r64), (b,b).
template <int CM>
__device__ __forceinline__ void pass_ores(const SysDesc& S, const Lanes& L, Dots<double>& d) {
  const DevMatrix& A = S.A;
  const Blk<double, kNS64> v{S.v64};
  const GatherSlot<double, kNS64> gx{S.v64 + IR_X * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    double* pc = v.chunk(c, L.lane);
    double ax = 0.0, bi = 0.0;
    if (in) { bi = __ldg(S.b + row); ax = __ldg(A.diag + row) * ldcg(pc + IR_X * kChunk); }
    ax = row_dot<double, true>(Cols<CM>::make(A, row), A.val, gx, A.diag, base, len, ax);
    if (in) {
      const double t = bi - ax;
      stcs(pc + IR_R * kChunk, t);
      d.add(0, t, t);
      d.add(1, bi, bi);
    }
  }
}

// P_OINIT: rhs32 = r64 / ||r64|| ; r32 = rhs32 ; u32 = M^-1 r32 ; d32 = 0.
__device__ __forceinline__ void pass_oinit(const SysDesc& S, const Lanes& L, double scale) {
  const Blk<double, kNS64> v64{S.v64};
  const Blk<float, kNS32> v32{S.v32};
  FOR_CHUNKS(S.A, L) {
    const int32_t row = c * kChunk + L.lane;
    if (row < S.A.n) {
      float* pc = v32.chunk(c, L.lane);
      const float rh = (float)(ldcs(v64.chunk(c, L.lane) + IR_R * kChunk) * scale);
      stcs(pc + V_RHS * kChunk, rh);
      stcs(pc + V_R * kChunk, rh);
      stcs(pc + V_U * kChunk, ldcs(pc + V_INVD * kChunk) * rh);
      stcs(pc + V_X * kChunk, 0.0f);
    }
  }
}

// P_OUNDO: x -= ||r64_prev|| * d32, taking back the last refinement step.
__device__ __forceinline__ void pass_oundo(const SysDesc& S, const Lanes& L, double rn_prev) {
  const Blk<double, kNS64> v64{S.v64};
  const Blk<float, kNS32> v32{S.v32};
  FOR_CHUNKS(S.A, L) {
    const int32_t row = c * kChunk + L.lane;
    if (row < S.A.n) {
      double* px = v64.chunk(c, L.lane) + IR_X * kChunk;
      *px = fma(-rn_prev, (double)ldcs(v32.chunk(c, L.lane) + V_X * kChunk), *px);
    }
  }
}

// P_OUPD: x += ||r64|| * d32 (FP64 solution accumulation).
__device__ __forceinline__ void pass_oupd(const SysDesc& S, const Lanes& L, double rn) {
  const Blk<double, kNS64> v64{S.v64};
  const Blk<float, kNS32> v32{S.v32};
  FOR_CHUNKS(S.A, L) {
    const int32_t row = c * kChunk + L.lane;
    if (row < S.A.n) {
      double* px = v64.chunk(c, L.lane) + IR_X * kChunk;
      *px = fma(rn, (double)ldcs(v32.chunk(c, L.lane) + V_X * kChunk), *px);
    }
  }
}

// ------------------------------- FP32 recurrences with FP64 reliable updates (FP32_RU) --
// x (FP64 block, slot x) holds the solution up to the last reliable update; d32 (FP32 block,
// slot d) the FP32 sum of alpha p since then.  A reliable update folds d32 into x, then
// recomputes the residual in FP64 and restarts the FP32 recurrences of r, u, w, s, q, z
// from it (p is kept, so the Krylov space is not restarted).

// t_x += A x and (DP) t_p += A p over one row's slots in one sweep: x in FP64 against the
// FP64 values, p in FP32 against the FP32 values.
template <bool DP, class CS>
__device__ __forceinline__ void row_dot_ures(const DevMatrix& A, const CS& col, const GatherSlot<double, kNS64>& gx,
                                             const GatherSlot<float, kNS32>& gp, int64_t base, int len, double& ax,
                                             float& ap) {
  int j = 0;
  for (; j + 8 <= len; j += 8) {
    int32_t c[8];
    double a[8];
    float b[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      c[k] = slot_col(col, base + (int64_t)(j + k) * kChunk, j + k);
      a[k] = ld_stream(A.val + base + (int64_t)(j + k) * kChunk);
      if (DP) b[k] = ld_stream(A.val32 + base + (int64_t)(j + k) * kChunk);
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      ax = fma(a[k], __ldg(A.diag + c[k]) * gx(c[k]), ax);
      if (DP) ap = fmaf(b[k], __ldg(A.diag32 + c[k]) * gp(c[k]), ap);
    }
  }
  int32_t c[7];
  double a[7];
  float b[7];
#pragma unroll
  for (int k = 0; k < 7; k++) {
    if (j + k < len) {
      c[k] = slot_col(col, base + (int64_t)(j + k) * kChunk, j + k);
      a[k] = ld_stream(A.val + base + (int64_t)(j + k) * kChunk);
      if (DP) b[k] = ld_stream(A.val32 + base + (int64_t)(j + k) * kChunk);
    }
  }
#pragma unroll
  for (int k = 0; k < 7; k++) {
    if (j + k < len) {
      ax = fma(a[k], __ldg(A.diag + c[k]) * gx(c[k]), ax);
      if (DP) ap = fmaf(b[k], __ldg(A.diag32 + c[k]) * gp(c[k]), ap);
    }
  }
}

// P_URES (d32 already folded into x).  x_zero: x = 0 (first update of a solve with x0 = 0);
// d_zero: d32 unset, set it to 0 (first update); p_zero: p = 0 (first update or a restart),
// so s = q = 0.
template <int CM>
__device__ __forceinline__ void pass_ures(const SysDesc& S, const Lanes& L, Dots<double>& d, bool x_zero,
                                          bool d_zero, bool p_zero) {
  const DevMatrix& A = S.A;
  const Blk<double, kNS64> v64{S.v64};
  const Blk<float, kNS32> v32{S.v32};
  const GatherSlot<double, kNS64> gx{S.v64 + IR_X * kChunk};
  const GatherSlot<float, kNS32> gp{S.v32 + V_P * kChunk};
  FOR_CHUNKS(A, L) {
    int64_t base; int len;
    chunk_slots<CM>(A, c, L.lane, base, len);
    const int32_t row = c * kChunk + L.lane;
    const bool in = row < A.n;
    float* p32 = v32.chunk(c, L.lane);
    double ax = 0.0, bi = 0.0;
    float ap = 0.0f, id = 0.0f;
    if (in) {
      bi = __ldg(S.b + row);
      id = ldcs(p32 + V_INVD * kChunk);
      if (!x_zero) ax = __ldg(A.diag + row) * ldcg(v64.chunk(c, L.lane) + IR_X * kChunk);
      if (!p_zero) ap = __ldg(A.diag32 + row) * ldcg(p32 + V_P * kChunk);
    }
    if (!x_zero) {
      if (p_zero) row_dot_ures<false>(A, Cols<CM>::make(A, row), gx, gp, base, len, ax, ap);
      else row_dot_ures<true>(A, Cols<CM>::make(A, row), gx, gp, base, len, ax, ap);
    }
    if (in) {
      const double t = bi - ax;
      const float r = (float)t;
      stcs(p32 + V_R * kChunk, r);
      stcs(p32 + V_U * kChunk, id * r);
      stcs(p32 + V_S * kChunk, ap);
      stcs(p32 + V_Q * kChunk, id * ap);
      if (d_zero) stcs(p32 + V_X * kChunk, 0.0f);
      d.add(0, t, t);
      d.add(1, bi, bi);
    }
  }
}

// P_UFLUSH: x += d32 ; d32 = 0.
__device__ __forceinline__ void pass_uflush(const SysDesc& S, const Lanes& L) {
  const Blk<double, kNS64> v64{S.v64};
  const Blk<float, kNS32> v32{S.v32};
  FOR_CHUNKS(S.A, L) {
    const int32_t row = c * kChunk + L.lane;
    if (row < S.A.n) {
      double* px = v64.chunk(c, L.lane) + IR_X * kChunk;
      float* pd = v32.chunk(c, L.lane) + V_X * kChunk;
      *px = *px + (double)*pd;
      *pd = 0.0f;
    }
  }
}

// ----------------------------------------------------------- partials and reduction --

// Block partials -> slot[0..3].  Every FP64 add costs a full warp instruction on the FP64
// pipe (about 16 SM cycles on this part), so the sum is organised to issue few of them.
// PACKED (sm holds (blockDim / 32) x 32 x 3 doubles): each lane stores its three partials;
// lane l of warp v (v < 3) adds value v of lane l over the warps; one shuffle tree per
// value.  Otherwise (sm holds 3 x 32 doubles): a shuffle tree in every warp, then warp 0
// sums the warps' results by a second tree.  Both orders are fixed: deterministic.
template <bool PACKED>
__device__ void write_block_partials(double a0, double a1, double a2, double* slot, double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if constexpr (PACKED) {
    double* mine = sm + (warp * 32 + lane) * 3;
    mine[0] = a0;
    mine[1] = a1;
    mine[2] = a2;
    __syncthreads();
    if (warp < 3) {
      double v = 0.0;
      for (int w = 0; w < nw; w++) v += sm[(w * 32 + lane) * 3 + warp];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
      if (lane == 0) slot[warp] = v;
      if (warp == 0 && lane == 0) slot[3] = 0.0;
    }
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_down_sync(kFull, a0, o);
      a1 += __shfl_down_sync(kFull, a1, o);
      a2 += __shfl_down_sync(kFull, a2, o);
    }
    if (lane == 0) { sm[warp * 3] = a0; sm[warp * 3 + 1] = a1; sm[warp * 3 + 2] = a2; }
    __syncthreads();
    if (warp == 0) {
      double s0 = lane < nw ? sm[lane * 3] : 0.0, s1 = lane < nw ? sm[lane * 3 + 1] : 0.0;
      double s2 = lane < nw ? sm[lane * 3 + 2] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(kFull, s0, o);
        s1 += __shfl_down_sync(kFull, s1, o);
        s2 += __shfl_down_sync(kFull, s2, o);
      }
      if (lane == 0) { slot[0] = s0; slot[1] = s1; slot[2] = s2; slot[3] = 0.0; }
    }
  }
}

// Sum the group's P partial slots in a fixed order; every CTA obtains identical bits.
__device__ void group_reduce(const double* part, int P, double* out) {
  // warp v (v < 3) sums value v over the P partial slots (lane-strided, then a shuffle
  // tree): three warps' worth of FP64 adds, the other warps idle.  Fixed order.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < 3) {
    double v = 0.0;
    for (int i = lane; i < P; i += 32) v += __ldcg(part + 4 * i + warp);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if (lane == 0) out[warp] = v;
    if (warp == 0 && lane == 0) out[3] = 0.0;
  }
  __syncthreads();
}

// ------------------------------------------------------------------------- control --

__device__ __forceinline__ void take_dots(Ctl& c) {
  c.gamma = c.red[0];
  c.delta = c.red[1];
  c.norm = sqrt(c.red[2]);
}

__device__ __forceinline__ bool passed(const Ctl& c, const SysDesc& S) {
  return S.norm == PPCG_NORM_PAPER_U_ABS ? (c.norm <= S.tol) : (c.norm <= S.tol * c.bnorm);
}

// Could the stopping test pass, given only gamma?  ||r||^2 <= dmax gamma is not needed: the
// lower bound dmin gamma <= ||r||^2 (REL_R) or gamma / dmax <= (u,u) (paper norm) decides
// "certainly not yet"; slack widens the window (used to predict the next iteration).
__device__ __forceinline__ bool may_pass(const Ctl& c, const SysDesc& S, double slack) {
  if (!(c.gamma >= 0.0)) return true;
  if (S.norm == PPCG_NORM_PAPER_U_ABS) return c.gamma / S.dmax <= slack * S.tol * S.tol;
  const double t = S.tol * c.bnorm;
  return c.gamma * S.dmin <= slack * t * t;
}

// alpha = gamma / den, with 1 / alpha and 1 / gamma for the next step, from one FP64
// division: r = 1 / (gamma den) gives 1 / den = gamma r and 1 / gamma = den r.  A division is
// a long dependent chain for the single thread that runs the control step, and the step is
// on every iteration's critical path, so the next step's beta = gamma / gamma_prev and
// beta gamma / alpha_prev become products with these inverses.  Where gamma den is near the
// ends of the FP64 range the three quotients are taken directly.
__device__ __forceinline__ void alpha_and_inverses(double gamma, double den, double& alpha, double& inv_alpha,
                                                   double& inv_gamma) {
  const double p = gamma * den;
  if (p > 1e-290 && p < 1e290) {
    const double r = 1.0 / p;
    alpha = gamma * (gamma * r);
    inv_gamma = den * r;
    inv_alpha = den * inv_gamma;
  } else {
    alpha = gamma / den;
    inv_alpha = den / gamma;
    inv_gamma = 1.0 / gamma;
  }
}

// The scalars of Alg. 2 (beta, then alpha).  Returns false on breakdown.
__device__ __forceinline__ bool scalars(Ctl& c, int it) {
  if (it > 0) {
    c.beta = c.gamma * c.inv_gamma;                    // gamma / gamma_prev
    double den = c.delta - (c.beta * c.gamma) * c.inv_alpha;   // delta - beta gamma / alpha_prev
    if (!(c.gamma > 0.0) || !(den > 0.0)) return false;
    alpha_and_inverses(c.gamma, den, c.alpha, c.inv_alpha, c.inv_gamma);
  } else {
    c.beta = 0.0;
    if (!(c.gamma > 0.0) || !(c.delta > 0.0)) return false;
    alpha_and_inverses(c.gamma, c.delta, c.alpha, c.inv_alpha, c.inv_gamma);
  }
  return true;
}

// The common step of the FP64 iteration -- S_AFTER_ITER, then S_TOP continuing with the
// next P_ITER -- on registers: the same operations in the same order as the general state
// machine below, committed only when every check of S_TOP lets the iteration continue;
// otherwise nothing is written and the general path takes the step.  (The control step is
// a serial chain run by one thread per CTA on every iteration; with the control block in
// shared memory each of its field accesses is a dependent round trip.)
// The same for the FP32_RU iteration step (S_U_AFTER_ITER, then S_U_TOP continuing).
__device__ __forceinline__ bool control_fast_ru(Ctl& c, const SysDesc& S, int iter_end) {
  const int iter = c.iter + 1, inner = c.inner_iter + 1;
  const double gamma_prev = c.gamma, alpha_prev = c.alpha;
  const double gamma = c.red[0], delta = c.red[1];
  const double norm = sqrt(c.red[2]);
  const double rmax = fmax(c.rmax, norm);
  if (iter >= iter_end) return false;
  if (!isfinite(gamma) || !isfinite(delta) || !isfinite(norm)) return false;
  if (c.last_rr_iter != iter) {
    const bool periodic = S.rr_period > 0 && iter - c.last_rr_iter >= S.rr_period;
    if (periodic || norm <= S.inner_tol * rmax || norm <= S.tol * c.bnorm || iter >= S.maxit) return false;
  }
  const double beta = gamma * c.inv_gamma;
  const double den = delta - (beta * gamma) * c.inv_alpha;
  if (!(gamma > 0.0) || !(den > 0.0)) return false;
  double alpha, inv_alpha, inv_gamma;
  alpha_and_inverses(gamma, den, alpha, inv_alpha, inv_gamma);
  c.inv_alpha = inv_alpha;
  c.inv_gamma = inv_gamma;
  c.gamma_prev = gamma_prev;
  c.alpha_prev = alpha_prev;
  c.iter = iter;
  c.inner_iter = inner;
  c.restart = 0;
  c.gamma = gamma;
  c.delta = delta;
  c.norm = norm;
  c.rmax = rmax;
  c.beta = beta;
  c.alpha = alpha;
  c.first = 0;
  c.pass = P_ITER;
  return true;
}

__device__ __forceinline__ bool control_fast(Ctl& c, const SysDesc& S, int iter_end) {
  if (c.state == S_U_AFTER_ITER) return control_fast_ru(c, S, iter_end);
  if (c.state != S_AFTER_ITER) return false;
  const int iter = c.iter + 1;
  const double gamma_prev = c.gamma, alpha_prev = c.alpha;
  const double gamma = c.red[0], delta = c.red[1];
  const int rr_valid = c.want_rr;
  const double norm = rr_valid ? sqrt(c.red[2]) : HUGE_VAL;
  const double bnorm = c.bnorm, tol = S.tol;
  const bool paper = S.norm == PPCG_NORM_PAPER_U_ABS;
  auto may = [&](double slack) {
    if (!(gamma >= 0.0)) return true;
    if (paper) return gamma / S.dmax <= slack * tol * tol;
    const double t = tol * bnorm;
    return gamma * S.dmin <= slack * t * t;
  };
  if (iter >= iter_end) return false;
  if (S.rr_period > 0 && iter % S.rr_period == 0 && c.last_rr_iter != iter) return false;
  if (S.gap_theta > 0.0 && gamma > 0.0 && gamma * S.gap_fall <= c.gamma_ref) return false;
  if (!rr_valid && may(1.001)) return false;
  if (paper ? (norm <= tol) : (norm <= tol * bnorm)) return false;
  if (iter >= S.maxit) return false;
  if (!isfinite(gamma) || !isfinite(delta)) return false;
  const double beta = gamma * c.inv_gamma;
  const double den = delta - (beta * gamma) * c.inv_alpha;
  if (!(gamma > 0.0) || !(den > 0.0)) return false;
  double alpha, inv_alpha, inv_gamma;
  alpha_and_inverses(gamma, den, alpha, inv_alpha, inv_gamma);
  const int want = may(64.0) ? 1 : 0;
  c.inv_alpha = inv_alpha;
  c.inv_gamma = inv_gamma;
  c.gamma_prev = gamma_prev;
  c.alpha_prev = alpha_prev;
  c.iter = iter;
  c.restart = 0;
  c.gamma = gamma;
  c.delta = delta;
  c.norm = norm;
  c.rr_valid = rr_valid;
  c.beta = beta;
  c.alpha = alpha;
  c.first = 0;
  c.want_rr = want;
  c.pass = P_ITER;
  return true;
}

// Thread 0 of every CTA: choose the next pass from the reduced partials of the last one.
__device__ void control(Ctl& c, const SysDesc& S, int iter_end) {
  if (control_fast(c, S, iter_end)) return;
  for (;;) {
    switch (c.state) {
      // ---- FP64 pipelined PCG
      case S_START:
        c.pass = P_SETUP1; c.state = S_AFTER_SETUP1; return;
      case S_AFTER_SETUP1:
        c.bnorm = sqrt(c.red[0]);
        if (S.norm == PPCG_NORM_REL_R && c.bnorm == 0.0) {   // A x = 0 -> x = 0
          c.status = PPCG_OK; c.pass = P_ZERO_X; c.state = S_FINAL; return;
        }
        c.pass = P_SETUP2; c.state = S_AFTER_SETUP2; return;
      case S_AFTER_SETUP2:
        take_dots(c); c.rr_valid = 1; c.gamma_ref = c.gamma; c.state = S_TOP; break;
      case S_AFTER_ITER:
        c.gamma_prev = c.gamma; c.alpha_prev = c.alpha; c.iter++; c.restart = 0;
        take_dots(c);
        c.rr_valid = c.want_rr;
        if (!c.want_rr) c.norm = HUGE_VAL;   // not accumulated this pass (see S_TOP)
        c.state = S_TOP; break;
      case S_AFTER_NORM:
        c.norm = sqrt(c.red[2]); c.rr_valid = 1; c.state = c.norm_return; break;
      case S_AFTER_RR2:
        take_dots(c); c.rr_valid = 1; c.rr_count++; c.last_rr_iter = c.iter; c.gamma_ref = c.gamma;
        if (passed(c, S)) { c.status = PPCG_OK; c.state = S_FINAL; break; }
        c.state = S_TOP; break;
      case S_TOP: {
        if (c.iter >= iter_end) { c.pass = P_NONE; c.exit_now = 1; return; }
        if (S.rr_period > 0 && c.iter > 0 && c.iter % S.rr_period == 0 && c.last_rr_iter != c.iter) {
          c.pass = P_RR1; c.state = S_AFTER_RR1; return;
        }
        // gamma has fallen by gap_fall since the residuals were last measured or replaced:
        // measure how far the recursive residual has drifted from b - A x
        if (S.gap_theta > 0.0 && c.iter > 0 && c.gamma > 0.0 && c.gamma * S.gap_fall <= c.gamma_ref) {
          c.pass = P_GAP; c.state = S_AFTER_GAP; return;
        }
        // ||r||^2 lies in [dmin, dmax] * gamma ((u,u) in gamma * [1/dmax, 1/dmin]); when the
        // last pass skipped the norm and the bound allows convergence, compute it exactly.
        if (!c.rr_valid && may_pass(c, S, 1.001)) {
          c.norm_return = S_TOP; c.pass = P_NORM; c.state = S_AFTER_NORM; return;
        }
        if (passed(c, S)) {
          if (S.norm == PPCG_NORM_PAPER_U_ABS) { c.status = PPCG_OK; c.state = S_FINAL; break; }
          c.pass = P_TRUE; c.state = S_AFTER_TRUE; return;
        }
        if (c.iter >= S.maxit) { c.status = PPCG_ERR_NOT_CONVERGED; c.state = S_FINAL; break; }
        if (!isfinite(c.gamma) || !isfinite(c.delta)) { c.status = PPCG_ERR_NONFINITE; c.state = S_FINAL; break; }
        if (!scalars(c, c.restart ? 0 : c.iter)) {
          if (c.iter > 0 && !c.restart && c.restarts < S.max_restarts) {
            // restart: replace the residuals, reset the direction recurrences, beta = 0 next
            c.restarts++; c.restart = 1;
            c.pass = P_RR1; c.state = S_AFTER_RR1; return;
          }
          c.status = PPCG_ERR_BREAKDOWN; c.state = S_FINAL; break;
        }
        c.first = (c.iter == 0 || c.restart);
        // accumulate the norm only where the next residual could be within 8x of the target
        c.want_rr = may_pass(c, S, 64.0) ? 1 : 0;
        c.pass = P_ITER; c.state = S_AFTER_ITER; return;
      }
      case S_AFTER_GAP:
        c.gamma_ref = c.gamma;
        if (sqrt(c.red[0]) > S.gap_theta * sqrt(c.red[1])) { c.pass = P_RR1; c.state = S_AFTER_RR1; return; }
        c.state = S_TOP; break;
      case S_AFTER_TRUE:
        c.res_true = sqrt(c.red[0]);
        if (c.res_true <= S.tol * c.bnorm) { c.status = PPCG_OK; c.state = S_DONE; c.pass = P_NONE; return; }
        c.pass = P_RR1; c.state = S_AFTER_RR1; return;
      case S_AFTER_RR1:
        c.pass = P_RR2; c.state = S_AFTER_RR2; return;
      case S_FINAL:
        if (!c.rr_valid) { c.norm_return = S_FINAL; c.pass = P_NORM; c.state = S_AFTER_NORM; return; }
        c.pass = P_TRUE; c.state = S_AFTER_FINAL; return;
      case S_AFTER_FINAL:
        c.res_true = sqrt(c.red[0]); c.state = S_DONE; c.pass = P_NONE; return;
      case S_DONE:
        c.pass = P_NONE; return;

      // ---- FP32 inner solves inside FP64 iterative refinement
      case S_O_START:
        c.pass = P_ORES; c.state = S_O_AFTER_ORES; return;
      case S_O_AFTER_ORES:
        c.rn = sqrt(c.red[0]);
        c.bnorm = sqrt(c.red[1]);
        c.res_true = c.rn;
        if (c.bnorm == 0.0) { c.status = PPCG_OK; c.pass = P_ZERO_X; c.state = S_O_AFTER_ZERO; return; }
        if (c.rn <= S.tol * c.bnorm) { c.status = PPCG_OK; c.state = S_DONE; c.pass = P_NONE; return; }
        if (!isfinite(c.rn)) { c.status = PPCG_ERR_NONFINITE; c.state = S_DONE; c.pass = P_NONE; return; }
        if (c.outer > 0 && !(c.rn <= 0.5 * c.rn_prev)) {
          // The FP32 inner solve did not halve the FP64 residual (kappa * eps32 near 1, or
          // recurrences that drifted): take the step back and finish with the FP64
          // iteration from the previous x.
          c.pass = P_OUNDO; c.state = S_O_AFTER_UNDO; return;
        }
        if (c.outer >= S.max_outer || c.iter >= S.maxit) {
          c.status = PPCG_ERR_NOT_CONVERGED; c.state = S_DONE; c.pass = P_NONE; return;
        }
        c.inner_target = fmax(S.inner_tol, 0.3 * S.tol * c.bnorm / c.rn);
        c.pass = P_OINIT; c.state = S_O_AFTER_OINIT; return;
      case S_O_AFTER_ZERO:
        c.res_true = 0.0; c.state = S_DONE; c.pass = P_NONE; return;
      case S_O_AFTER_OINIT:
        c.inner_iter = 0; c.last_rr_iter = -1; c.restart = 0; c.restarts = 0; c.rr_norm_prev = 0.0;
        c.pass = P_SETUP2; c.state = S_I_AFTER_SETUP2; return;
      case S_I_AFTER_SETUP2:
        take_dots(c); c.inner_norm0 = c.norm; c.state = S_I_TOP; break;
      case S_I_AFTER_ITER:
        c.gamma_prev = c.gamma; c.alpha_prev = c.alpha; c.iter++; c.inner_iter++; c.restart = 0;
        take_dots(c); c.state = S_I_TOP; break;
      case S_I_AFTER_RR2:
        take_dots(c); c.rr_count++; c.last_rr_iter = c.inner_iter;
        if (!c.restart && !(c.norm <= 4.0 * c.rr_norm_prev)) {
          // periodic replacement: the true inner residual came out more than 4x the recursive
          // one it replaced -- the FP32 recurrences have drifted; end this inner solve.
          c.pass = P_OUPD; c.state = S_O_AFTER_OUPD; return;
        }
        c.state = S_I_TOP; break;
      case S_I_AFTER_RR1:
        c.pass = P_RR2; c.state = S_I_AFTER_RR2; return;
      case S_I_TOP: {
        if (c.iter >= iter_end) { c.pass = P_NONE; c.exit_now = 1; return; }
        if (!isfinite(c.gamma) || !isfinite(c.delta) || !isfinite(c.norm)) {
          // the FP32 inner solve overflowed: x still holds the last good refinement
          c.state = S_O_AFTER_UNDO; break;
        }
        if (c.norm <= c.inner_target * c.inner_norm0 || c.inner_iter >= S.inner_maxit || c.iter >= S.maxit) {
          c.pass = P_OUPD; c.state = S_O_AFTER_OUPD; return;
        }
        if (S.rr_period > 0 && c.inner_iter > 0 && c.inner_iter % S.rr_period == 0 &&
            c.last_rr_iter != c.inner_iter) {
          c.rr_norm_prev = c.norm;   // recursive residual being replaced
          c.pass = P_RR1; c.state = S_I_AFTER_RR1; return;
        }
        if (!scalars(c, c.restart ? 0 : c.inner_iter)) {
          if (c.inner_iter == 0) { c.status = PPCG_ERR_BREAKDOWN; c.state = S_DONE; c.pass = P_NONE; return; }
          if (!c.restart && c.restarts < S.max_restarts) {
            // restart the inner recurrences from the current correction (as in FP64)
            c.restarts++; c.restart = 1;
            c.pass = P_RR1; c.state = S_I_AFTER_RR1; return;
          }
          c.pass = P_OUPD; c.state = S_O_AFTER_OUPD; return;   // keep the correction so far
        }
        c.first = (c.inner_iter == 0 || c.restart);
        c.pass = P_ITER; c.state = S_I_AFTER_ITER; return;
      }
      case S_O_AFTER_UNDO:
        // FP64 iteration from x: its first step starts the recurrences afresh (beta = 0)
        c.fallback = 1; c.restart = 1; c.restarts = 0; c.last_rr_iter = -1;
        c.status = PPCG_ERR_NOT_CONVERGED;
        c.state = S_START; break;
      case S_O_AFTER_OUPD:
        c.outer++; c.rn_prev = c.rn;
        c.pass = P_ORES; c.state = S_O_AFTER_ORES; return;

      // ---- FP32 recurrences with FP64 reliable updates.  An update is due every rr_period
      // iterations and when the recursive residual has fallen by inner_tol from its largest
      // value since the last one, and is forced when the recursive residual passes the
      // stopping test or maxit is reached; the FP64 residual it computes decides.
      case S_U_START:
        c.pass = P_URES; c.state = S_U_AFTER_RES; return;
      case S_U_AFTER_FLUSH:
        c.pass = P_URES; c.state = S_U_AFTER_RES; return;
      case S_U_AFTER_RES: {
        const double rt = sqrt(c.red[0]);
        const bool first = c.outer == 0;
        if (first) c.bnorm = sqrt(c.red[1]);
        c.outer++;
        if (c.bnorm == 0.0) { c.status = PPCG_OK; c.pass = P_ZERO_X; c.state = S_O_AFTER_ZERO; return; }
        if (!isfinite(rt)) {
          if (first) { c.status = PPCG_ERR_NONFINITE; c.res_true = rt; c.state = S_DONE; c.pass = P_NONE; return; }
          c.state = S_O_AFTER_UNDO; break;   // FP64 iteration from x
        }
        if (!first && c.ru_due) {
          // A stall: the FP32 recursion claimed at least a 4x fall since the last update
          // and the FP64 residual did not even halve.  Three in a row: FP32 cannot make
          // progress on this system (kappa * eps32 too large).
          if (rt <= 0.5 * c.rn) c.stalls = 0;
          else if (c.rr_norm_prev <= 0.25 * c.rn) c.stalls++;
          if (c.stalls >= 3) { c.state = S_O_AFTER_UNDO; break; }
        }
        c.ru_due = 0;
        c.rn_prev = c.rn; c.rn = rt; c.res_true = rt;
        if (rt <= S.tol * c.bnorm || c.iter >= S.maxit) {   // x already holds every step
          c.status = rt <= S.tol * c.bnorm ? PPCG_OK : PPCG_ERR_NOT_CONVERGED;
          c.state = S_DONE; c.pass = P_NONE; return;
        }
        c.last_rr_iter = c.iter;
        c.pass = first ? P_SETUP2 : P_URR2; c.state = S_U_AFTER_RR2; return;
      }
      case S_U_AFTER_RR2:
        take_dots(c);
        if (c.outer > 1) c.rr_count++;
        c.rmax = c.norm;
        c.state = S_U_TOP; break;
      case S_U_AFTER_ITER:
        c.gamma_prev = c.gamma; c.alpha_prev = c.alpha; c.iter++; c.inner_iter++; c.restart = 0;
        take_dots(c);
        c.rmax = fmax(c.rmax, c.norm);
        c.state = S_U_TOP; break;
      case S_U_TOP: {
        if (c.iter >= iter_end) { c.pass = P_NONE; c.exit_now = 1; return; }
        if (!isfinite(c.gamma) || !isfinite(c.delta) || !isfinite(c.norm)) { c.state = S_O_AFTER_UNDO; break; }
        if (c.last_rr_iter != c.iter) {
          const bool periodic = S.rr_period > 0 && c.iter - c.last_rr_iter >= S.rr_period;
          if (periodic || c.norm <= S.inner_tol * c.rmax || c.norm <= S.tol * c.bnorm || c.iter >= S.maxit) {
            c.ru_due = 1; c.rr_norm_prev = c.norm;
            c.pass = P_UFLUSH; c.state = S_U_AFTER_FLUSH; return;
          }
        }
        if (!scalars(c, c.restart ? 0 : c.inner_iter)) {
          if (c.inner_iter > 0 && !c.restart && c.restarts < S.max_restarts) {
            c.restarts++; c.restart = 1; c.ru_due = 0;   // update with p = 0: next beta = 0
            c.pass = P_UFLUSH; c.state = S_U_AFTER_FLUSH; return;
          }
          if (c.inner_iter == 0) {
            c.status = PPCG_ERR_BREAKDOWN; c.pass = P_TRUE; c.state = S_AFTER_FINAL; return;
          }
          c.state = S_O_AFTER_UNDO; break;   // restarts used up: FP64 iteration from x
        }
        c.first = (c.inner_iter == 0 || c.restart);
        c.pass = P_ITER; c.state = S_U_AFTER_ITER; return;
      }
      default:
        c.status = PPCG_ERR_ARG; c.state = S_DONE; c.pass = P_NONE; return;
    }
  }
}

// ------------------------------------ matrix-free constant-coefficient box stencil --
// When A = cd I + co (adjacency of the (2R+1)^3 box on a g^3 grid, truncated at the
// boundary) -- the 125-point Poisson family of Table II for R = 2 -- a product A v needs no
// matrix: the box sum B(v)_i (v summed over row i's box, i included) is taken axis by axis.
// Stage X writes t1 = the x-sums of v, stage Y writes t2 = the y-sums of t1, and the
// consuming pass adds the z-sums of t2.  Rows are in grid order (x fastest), so each stage
// reads its 2R+1 neighbours at fixed row offsets (1, g, g^2): for a warp, contiguous 32-row
// runs.  Stage Y and the iteration pass march along their axis with a running window sum
// (box_march), so per product and row the sums cost 2R + 4 FP64 adds (interior rows, plus
// a direct window at each segment start) and 4 intermediate streams instead of
// (2R+1)^3 - 1 FMAs and the matrix stream.  The FP64 pipe, not HBM, bounds these passes.
// Then (A v)_i = cd v_i + co (B_i - v_i) and (A D^-1 v)_i = v_i + (co / cd) (B_i - v_i).

__device__ __forceinline__ void box_coords(int32_t row, int32_t g, int32_t& z, int32_t& y, int32_t& x) {
  const int32_t zy = row / g;
  x = row - zy * g;
  z = zy / g;
  y = zy - z * g;
}

// Window sum along one axis: the sum of f(row + d * stride) over the offsets d in [-R, R]
// that stay on the grid (0 <= c + d < g, c the row's coordinate on that axis), added in
// ascending d with the first term taken as is -- no 0.0 start, so a window of w terms costs
// w - 1 FP64 adds, the pipe that bounds these passes.  The interior of the R = 2 family
// (Table II) is unrolled; every form adds the same terms in the same order.
template <class F>
__device__ __forceinline__ double axis_sum(const F& f, int32_t row, int32_t c, int32_t g, int32_t R,
                                           int64_t stride) {
  if (R == 2 && c >= 2 && c + 2 < g) {
    const double a0 = f(row - 2 * stride), a1 = f(row - stride), a2 = f(row), a3 = f(row + stride),
                 a4 = f(row + 2 * stride);
    return (((a0 + a1) + a2) + a3) + a4;
  }
  const int32_t lo = max(-R, -c), hi = min(R, g - 1 - c);
  double s = f(row + lo * stride);
  for (int32_t d = lo + 1; d <= hi; d++) s += f(row + d * stride);
  return s;
}

struct LoadCg {
  const double* p;
  __device__ __forceinline__ double operator()(int64_t j) const { return __ldcg(p + j); }
};
struct LoadSlot {
  GatherSlot<double, kNS64> g;
  __device__ __forceinline__ double operator()(int64_t j) const { return g((int32_t)j); }
};

// Stage X for one or two FP64-block slots (slot_b < 0: one).
__device__ void box_stage_x(const SysDesc& S, const Lanes& L, int slot_a, int slot_b) {
  const int32_t n = (int32_t)S.A.n, g = S.box_g, R = S.box_r;
  const LoadSlot va{{S.v64 + slot_a * kChunk}};
  const LoadSlot vb{{S.v64 + (slot_b < 0 ? slot_a : slot_b) * kChunk}};
  double* t1a = S.box_t;
  double* t1b = S.box_t + n;
  FOR_CHUNKS(S.A, L) {
    const int32_t row = c * kChunk + L.lane;
    if (row >= n) continue;
    int32_t z, y, x;
    box_coords(row, g, z, y, x);
    __stcg(t1a + row, axis_sum(va, row, x, g, R, 1));
    if (slot_b >= 0) __stcg(t1b + row, axis_sum(vb, row, x, g, R, 1));
  }
}

// Marching split of a stage along y or z: work items (in-plane position, segment), the
// segment a run of `len` consecutive positions along the axis.  The first position of a
// segment takes its window directly (axis_sum); each next one updates the running window
// sum by the entering and the leaving term -- 2 FP64 adds per row instead of 2R.  Segments
// are at least 8 long (fewer items than threads on small grids) and otherwise as many as
// the group's threads can take at once.  Item t: segment t / g^2, in-plane index t % g^2
// with x fastest, so the lanes of a warp hold consecutive rows.
struct BoxMarch {
  int32_t nseg, len;
};
// The group's warps in CTA-interleaved order (warp w of CTA r -> w * ranks + r), so that
// when the marching items fill only part of the group the idle warps are spread over every
// SM instead of being the last CTAs' (185^3: 136,900 items for 151,552 threads; with the
// plain order ~15 SMs had no work in the marching stages).
__device__ __forceinline__ int64_t box_item0(const Lanes& L) {
  const int32_t nw = (int32_t)(blockDim.x >> 5), r = L.gw / nw, w = L.gw - r * nw;
  return ((int64_t)w * (L.W / nw) + r) * 32 + L.lane;
}
__device__ __forceinline__ BoxMarch box_march(int32_t g, int32_t threads) {
  const int32_t plane = g * g;
  int32_t nseg = min((g + 7) / 8, threads / plane);
  if (nseg < 1) nseg = 1;
  const int32_t len = (g + nseg - 1) / nseg;
  return {(g + len - 1) / len, len};
}

// The running window sum along an axis (stride `st` rows) moved from position p - 1 to p:
// add the entering term (p + R on the grid), subtract the leaving one (p - R - 1).
__device__ __forceinline__ double window_step(const double* t, int64_t row, int32_t p, int32_t g, int32_t R,
                                              int64_t st, double s) {
  if (p + R < g) s += __ldcg(t + row + R * st);
  if (p - R - 1 >= 0) s -= __ldcg(t + row - (R + 1) * st);
  return s;
}

// Stage Y: t2 = y-sums of t1 (one or two arrays), marching along y.
__device__ void box_stage_y(const SysDesc& S, const Lanes& L, bool two) {
  const int32_t n = (int32_t)S.A.n, g = S.box_g, R = S.box_r;
  const double* t1a = S.box_t;
  const double* t1b = S.box_t + n;
  double* t2a = S.box_t + 2 * (int64_t)n;
  double* t2b = S.box_t + 3 * (int64_t)n;
  const int32_t plane = g * g;
  const BoxMarch m = box_march(g, L.W * 32);
  const int32_t items = m.nseg * plane;
  for (int64_t t = box_item0(L); t < items; t += (int64_t)L.W * 32) {
    const int32_t seg = (int32_t)(t / plane), rem = (int32_t)(t - (int64_t)seg * plane);
    const int32_t z = rem / g, x = rem - z * g;
    const int32_t y0 = seg * m.len, y1 = min(g, y0 + m.len);
    int64_t row = (int64_t)z * plane + (int64_t)y0 * g + x;
    double sa = axis_sum(LoadCg{t1a}, row, y0, g, R, g);
    double sb = two ? axis_sum(LoadCg{t1b}, row, y0, g, R, g) : 0.0;
    __stcg(t2a + row, sa);
    if (two) __stcg(t2b + row, sb);
    for (int32_t y = y0 + 1; y < y1; y++) {
      row += g;
      sa = window_step(t1a, row, y, g, R, g, sa);
      __stcg(t2a + row, sa);
      if (two) {
        sb = window_step(t1b, row, y, g, R, g, sb);
        __stcg(t2b + row, sb);
      }
    }
  }
}

// z-sums of t2 (array k = 0 or 1) for one row: the box sum B_row.
__device__ __forceinline__ double box_z(const SysDesc& S, int32_t row, int32_t z, int k) {
  const int32_t n = (int32_t)S.A.n, g = S.box_g, R = S.box_r;
  const LoadCg t2{S.box_t + (2 + k) * (int64_t)n};
  return axis_sum(t2, row, z, g, R, (int64_t)g * g);
}

// Sources of the box stages for an FP64 pass (slot_a < 0: the pass needs no product).
__device__ __forceinline__ void box_sources(const Ctl& C, const SysDesc& S, int& slot_a, int& slot_b) {
  slot_a = slot_b = -1;
  switch (C.pass) {
    case P_SETUP1: if (!(S.x_zero != 0 && !C.fallback)) slot_a = V_X; break;
    case P_SETUP2: slot_a = V_R; break;
    case P_ITER: slot_a = (C.iter & 1) ? V_WB : V_WA; break;
    case P_TRUE: case P_GAP: slot_a = V_X; break;
    case P_RR1: slot_a = V_X; if (!(C.iter == 0 || C.restart)) slot_b = V_P; break;
    case P_RR2: slot_a = V_R; slot_b = V_S; break;
    default: break;
  }
}

// The FP64 passes with the box product (the other passes are shared with the SELL path).
// Returns whether the pass produced partials.
__device__ bool box_pass(const SysDesc& S, const Ctl& C, const Lanes& L, Dots<double>& d, bool paper) {
  const int32_t n = (int32_t)S.A.n, g = S.box_g;
  const double cd = S.box_cd, co = S.box_co, ch = S.box_co / S.box_cd;
  const Blk<double, kNS64> v{S.v64};
  switch (C.pass) {
    case P_SETUP1:
    case P_TRUE:
    case P_GAP:
    case P_RR1: {
      const bool x_zero = C.pass == P_SETUP1 && S.x_zero != 0 && !C.fallback;
      const bool rr = C.pass == P_RR1, p_zero = rr && (C.iter == 0 || C.restart);
      FOR_CHUNKS(S.A, L) {
        const int32_t row = c * kChunk + L.lane;
        if (row >= n) continue;
        int32_t z, y, x;
        box_coords(row, g, z, y, x);
        double* pc = v.chunk(c, L.lane);
        const double bi = __ldg(S.b + row);
        double ax = 0.0;
        if (!x_zero) {
          const double xi = ldcg(pc + V_X * kChunk);
          ax = fma(co, box_z(S, row, z, 0) - xi, cd * xi);
        }
        const double ri = bi - ax;
        if (C.pass == P_TRUE) { d.add(0, ri, ri); continue; }
        if (C.pass == P_GAP) {
          const double rr_i = ldcs(pc + V_R * kChunk), gi = ri - rr_i;
          d.add(0, gi, gi);
          d.add(1, rr_i, rr_i);
          continue;
        }
        const double id = ldcs(pc + V_INVD * kChunk);
        stcs(pc + V_R * kChunk, ri);
        stcs(pc + V_U * kChunk, id * ri);
        if (rr) {
          double ap = 0.0;
          if (!p_zero) {
            const double pi = ldcg(pc + V_P * kChunk);
            ap = fma(co, box_z(S, row, z, 1) - pi, cd * pi);
          }
          stcs(pc + V_S * kChunk, ap);
          stcs(pc + V_Q * kChunk, id * ap);
        } else {
          d.add(0, bi, bi);
          d.add(1, ri, ri);
        }
      }
      return !rr;
    }
    case P_SETUP2:
    case P_RR2: {
      const bool rr = C.pass == P_RR2;
      const int wcs = rr && (C.iter & 1) ? V_WB : V_WA;
      FOR_CHUNKS(S.A, L) {
        const int32_t row = c * kChunk + L.lane;
        if (row >= n) continue;
        int32_t z, y, x;
        box_coords(row, g, z, y, x);
        double* pc = v.chunk(c, L.lane);
        const double ri = ldcg(pc + V_R * kChunk), ui = ldcs(pc + V_U * kChunk);
        const double wi = fma(ch, box_z(S, row, z, 0) - ri, ri);
        stcs(pc + wcs * kChunk, wi);
        if (rr) {
          const double si = ldcg(pc + V_S * kChunk);
          stcs(pc + V_Z * kChunk, fma(ch, box_z(S, row, z, 1) - si, si));
        }
        d.add(0, ri, ui);
        d.add(1, wi, ui);
        if (paper) d.add(2, ui, ui); else d.add(2, ri, ri);
      }
      return true;
    }
    case P_ITER: {
      const bool first = C.first != 0, with_rr = C.want_rr != 0;
      const double alpha = C.alpha, beta = C.beta;
      const int wcs = (C.iter & 1) ? V_WB : V_WA;
      const int wns = (C.iter & 1) ? V_WA : V_WB;
      // Rows in marching order along z (see box_march): the z-window of t2 is carried from
      // one row to the next of the segment.
      const int32_t R = S.box_r, plane = g * g;
      const double* t2 = S.box_t + 2 * (int64_t)n;
      const BoxMarch m = box_march(g, L.W * 32);
      const int32_t items = m.nseg * plane;
      for (int64_t t = box_item0(L); t < items; t += (int64_t)L.W * 32) {
        const int32_t seg = (int32_t)(t / plane), rem = (int32_t)(t - (int64_t)seg * plane);
        const int32_t z0 = seg * m.len, z1 = min(g, z0 + m.len);
        int32_t row = z0 * plane + rem;
        double bs = axis_sum(LoadCg{t2}, row, z0, g, R, plane);
        for (int32_t z = z0;;) {
          double* pc = v.chunk(row / kChunk, row % kChunk);
          const double wi = ldcg(pc + wcs * kChunk);
          // n_i = (A M^-1 w)_i = w_i + (co / cd) (B(w)_i - w_i)
          const double ni = fma(ch, bs - wi, wi);
          const double id = ldcs(pc + V_INVD * kChunk), ui = ldcs(pc + V_U * kChunk);
          const double mi = id * wi;
          const double zi = first ? ni : fma(beta, ldcs(pc + V_Z * kChunk), ni);
          const double qi = first ? mi : fma(beta, ldcs(pc + V_Q * kChunk), mi);
          const double si = first ? wi : fma(beta, ldcs(pc + V_S * kChunk), wi);
          const double pi = first ? ui : fma(beta, ldcs(pc + V_P * kChunk), ui);
          const double xi = fma(alpha, pi, ldcs(pc + V_X * kChunk));
          const double ri = fma(-alpha, si, ldcs(pc + V_R * kChunk));
          const double un = fma(-alpha, qi, ui);
          const double wnn = fma(-alpha, zi, wi);
          stcs(pc + V_Z * kChunk, zi);
          stcs(pc + V_Q * kChunk, qi);
          stcs(pc + V_S * kChunk, si);
          stcs(pc + V_P * kChunk, pi);
          stcs(pc + V_X * kChunk, xi);
          stcs(pc + V_R * kChunk, ri);
          stcs(pc + V_U * kChunk, un);
          stcs(pc + wns * kChunk, wnn);
          d.add(0, ri, un);
          d.add(1, wnn, un);
          if (with_rr) { if (paper) d.add(2, un, un); else d.add(2, ri, ri); }
          if (++z >= z1) break;
          row += plane;
          bs = window_step(t2, row, z, g, R, plane, bs);
        }
      }
      return true;
    }
    default:
      return false;
  }
}

// ------------------------------------------------------------------------- driver --

// Shared state of run_system.  The grid path keeps the per-warp-tree block reduction and a
// small buffer (its 2 x 512-thread CTAs per SM want the L1 for gathers and spills; a 12 KB
// buffer measured 3% slower at 256^3); the 256-thread cluster path packs its adds.
template <int NSM> struct SharedT {
  static constexpr bool kPacked = NSM > 3 * 32;
  SysDesc S;
  Ctl C;
  double sm[NSM];
  double part[2][4];   // cluster path: this CTA's block partials, read by the whole cluster
};

// Cluster path: the cluster's block partials, read from every CTA's shared memory by lanes
// 0..nranks-1 of warp 0 and summed by a fixed shuffle tree (deterministic for a given
// cluster size, a power of two up to 16).  out is written by thread 0.
__device__ __forceinline__ void cluster_reduce(const double* part, double* out) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int nr = (int)cluster_nranks();
    const uint32_t base = smem_addr(part);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    if (lane < nr) {
      s0 = ld_dsmem(base, lane);
      s1 = ld_dsmem(base + 8, lane);
      s2 = ld_dsmem(base + 16, lane);
    }
    for (int o = nr / 2; o > 0; o >>= 1) {
      s0 += __shfl_down_sync(kFull, s0, o);
      s1 += __shfl_down_sync(kFull, s1, o);
      s2 += __shfl_down_sync(kFull, s2, o);
    }
    if (lane == 0) { out[0] = s0; out[1] = s1; out[2] = s2; out[3] = 0.0; }
  }
}
constexpr int kSmGrid = 3 * 32, kSmCluster = 3 * 32 * (kClusterThreads / 32);

// BOX: the kernel carries the matrix-free box passes (a plan with box_g > 0 runs only on
// such a kernel, every other plan only on the others, so the SELL kernels' register
// allocation does not carry the box code); a mismatch ends the solve with PPCG_ERR_ARG.
// CM: the column mode -- kColA: every pass reads the 4-byte columns; kColDict: the iteration
// passes read the column dictionary (a plan without one ends with PPCG_ERR_ARG); kColPat:
// every SELL pass forms its columns from the offset pattern (a plan without one ends with
// PPCG_ERR_ARG).  A pattern matrix is also a valid SELL matrix, so kColA kernels run it too.
// PF: the FP64 iteration pass prefetches each chunk's own entries into L2 (see pass_iter).
template <bool STAGED, bool BOX = false, int CM = kColA, bool PF = false, class G, class Shared>
__device__ void run_system(G& g, const SysDesc* Sg, int budget, Shared& sh, unsigned char* stage_mem,
                           uint64_t* stage_bars, unsigned& phases) {
  __syncthreads();   // previous system's readers of sh are done
  if (threadIdx.x == 0) {
    sh.S = *Sg;
    // the control block was written by an earlier launch or kernel: read it through L2
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(sh.S.ctl);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sh.C);
    for (int i = 0; i < (int)(sizeof(Ctl) / 8); i++) dst[i] = __ldcg(src + i);
    if (sh.C.t_start == 0) sh.C.t_start = globaltimer();
    sh.C.exit_now = 0;
    if ((sh.S.box_g > 0) != BOX || (CM == kColDict && !sh.S.A.cidx) || (CM == kColPat && sh.S.A.pat_k <= 0)) {
      sh.C.status = PPCG_ERR_ARG;
      sh.C.state = S_DONE;
    }
  }
  __syncthreads();
  const SysDesc& S = sh.S;
  Ctl& C = sh.C;
  if (S.budget > 0) budget = S.budget;     // per-system epoch budget (server)
  const int iter_end = budget > 0 && C.iter < 0x7fffffff - budget ? C.iter + budget : 0x7fffffff;
  const int nw = blockDim.x >> 5;
  Lanes L;
  L.lane = threadIdx.x & 31;
  L.gw = g.rank() * nw + (threadIdx.x >> 5);
  L.W = g.size() * nw;
  const bool paper = S.norm == PPCG_NORM_PAPER_U_ABS;
  const int P = g.size();
  constexpr bool kPacked = Shared::kPacked;
  constexpr int CMO = CM == kColDict ? kColA : CM;   // column mode of the passes other than P_ITER

  for (;;) {
    if (threadIdx.x == 0) control(C, S, iter_end);
    __syncthreads();
    const int pass = C.pass;
    if (pass == P_NONE) break;
    const bool fp32 = S.precision != PPCG_FP64 && (C.state >= S_O_START);
    double* slot = G::kCluster ? &sh.part[C.parity][0] : S.part + ((size_t)C.parity * P + g.rank()) * 4;
    bool partials = true;
    if (!fp32 && S.variant == PPCG_VARIANT_JACOBI_SCALED) {
      Dots<double> d;
      switch (pass) {
        case P_SETUP1: spass_setup1<CMO>(S, L, d, S.x_zero != 0); break;
        case P_SETUP2: spass_setup2<CMO>(S, L, d, paper); break;
        case P_ITER:
          if (C.first) spass_iter<true, CMO>(S, L, d, C.alpha, C.beta, C.iter, paper, C.want_rr != 0);
          else spass_iter<false, CMO>(S, L, d, C.alpha, C.beta, C.iter, paper, C.want_rr != 0);
          break;
        case P_NORM: spass_norm(S, L, d, paper); break;
        case P_TRUE: spass_true<CMO>(S, L, d); break;
        case P_GAP: spass_gap<CMO>(S, L, d); break;
        case P_RR1: spass_rr1<CMO>(S, L, C.iter == 0 || C.restart); partials = false; break;
        case P_RR2: spass_rr2<CMO>(S, L, d, C.iter, paper); break;
        case P_ZERO_X: pass_zero_x<kNSS, VS_X>(S, L); partials = false; break;
        default: partials = false; break;
      }
      if (partials) write_block_partials<kPacked>(d.get(0), d.get(1), d.get(2), slot, sh.sm);
    } else if (BOX && !fp32 && (pass == P_SETUP1 || pass == P_SETUP2 || pass == P_ITER ||
                                          pass == P_TRUE || pass == P_GAP || pass == P_RR1 || pass == P_RR2)) {
      int sa, sb;
      box_sources(C, S, sa, sb);
      if (sa >= 0) {
        box_stage_x(S, L, sa, sb);
        if (!g.sync()) { if (threadIdx.x == 0) { C.status = PPCG_ERR_TIMEOUT; C.state = S_DONE; } break; }
        box_stage_y(S, L, sb >= 0);
        if (!g.sync()) { if (threadIdx.x == 0) { C.status = PPCG_ERR_TIMEOUT; C.state = S_DONE; } break; }
      }
      Dots<double> d;
      partials = box_pass(S, C, L, d, paper);
      if (partials) write_block_partials<kPacked>(d.get(0), d.get(1), d.get(2), slot, sh.sm);
    } else if (!fp32) {
      Dots<double> d;
      const View<double, kNS64> V = view64(S);
      switch (pass) {
        case P_SETUP1: pass_setup1<CMO>(S, L, d, S.x_zero != 0 && !C.fallback); break;
        case P_SETUP2: pass_setup2<double, kNS64, CMO>(S.A, V, L, d, paper); break;
        case P_ITER:
          if (STAGED) {
            unsigned char* wst = stage_mem + (threadIdx.x >> 5) * kWarpStageBytes;
            uint64_t* bars = stage_bars + 2 * (threadIdx.x >> 5);
            if (C.first) pass_iter_staged<double, kNS64, true>(S.A, V, L, d, C.alpha, C.beta, C.iter, paper, wst, bars, phases, S.err);
            else pass_iter_staged<double, kNS64, false>(S.A, V, L, d, C.alpha, C.beta, C.iter, paper, wst, bars, phases, S.err);
          } else {
            if (C.first) pass_iter<double, kNS64, true, CM>(S.A, V, L, d, C.alpha, C.beta, C.iter, paper, C.want_rr != 0, PF);
            else pass_iter<double, kNS64, false, CM>(S.A, V, L, d, C.alpha, C.beta, C.iter, paper, C.want_rr != 0, PF);
          }
          break;
        case P_TRUE: pass_true<kNS64, V_X, CMO>(S, L, d); break;
        case P_GAP: pass_gap<kNS64, V_X, V_R, CMO>(S, L, d); break;
        case P_NORM: pass_norm(S.A, V, L, d, paper); break;
        case P_RR1: pass_rr1<double, kNS64, CMO>(S.A, V, L, C.iter == 0 || C.restart); partials = false; break;
        case P_RR2: pass_rr2<double, kNS64, CMO>(S.A, V, L, d, C.iter, paper); break;
        case P_ZERO_X: pass_zero_x<kNS64, V_X>(S, L); partials = false; break;
        default: partials = false; break;
      }
      if (partials) write_block_partials<kPacked>(d.get(0), d.get(1), d.get(2), slot, sh.sm);
    } else if (pass == P_ORES || pass == P_ZERO_X || pass == P_OINIT || pass == P_OUPD || pass == P_OUNDO ||
               pass == P_URES || pass == P_UFLUSH) {
      Dots<double> d;
      switch (pass) {
        case P_URES:
          pass_ures<CMO>(S, L, d, S.x_zero != 0 && C.outer == 0, C.outer == 0, C.inner_iter == 0 || C.restart);
          break;
        case P_UFLUSH: pass_uflush(S, L); partials = false; break;
        case P_ORES: pass_ores<CMO>(S, L, d); break;
        case P_ZERO_X: pass_zero_x<kNS64, IR_X>(S, L); partials = false; break;
        case P_OINIT: pass_oinit(S, L, 1.0 / C.rn); partials = false; break;
        case P_OUPD: pass_oupd(S, L, C.rn); partials = false; break;
        case P_OUNDO: pass_oundo(S, L, C.rn_prev); partials = false; break;
        default: partials = false; break;
      }
      if (partials) write_block_partials<kPacked>(d.get(0), d.get(1), d.get(2), slot, sh.sm);
    } else {
      Dots<float> d;
      const View<float, kNS32> V = view32(S);
      switch (pass) {
        case P_SETUP2: pass_setup2<float, kNS32, CMO>(S.A, V, L, d, paper); break;
        case P_ITER:
          if (STAGED) {
            unsigned char* wst = stage_mem + (threadIdx.x >> 5) * kWarpStageBytes;
            uint64_t* bars = stage_bars + 2 * (threadIdx.x >> 5);
            if (C.first) pass_iter_staged<float, kNS32, true>(S.A, V, L, d, (float)C.alpha, (float)C.beta, C.inner_iter, paper, wst, bars, phases, S.err);
            else pass_iter_staged<float, kNS32, false>(S.A, V, L, d, (float)C.alpha, (float)C.beta, C.inner_iter, paper, wst, bars, phases, S.err);
          } else {
            if (C.first) pass_iter<float, kNS32, true, CM>(S.A, V, L, d, (float)C.alpha, (float)C.beta, C.inner_iter, paper);
            else pass_iter<float, kNS32, false, CM>(S.A, V, L, d, (float)C.alpha, (float)C.beta, C.inner_iter, paper);
          }
          break;
        case P_RR1: pass_rr1<float, kNS32, CMO>(S.A, V, L, C.inner_iter == 0 || C.restart); partials = false; break;
        case P_RR2: pass_rr2<float, kNS32, CMO>(S.A, V, L, d, C.inner_iter, paper); break;
        case P_URR2: pass_rr2<float, kNS32, CMO>(S.A, V, L, d, C.inner_iter, paper); break;
        default: partials = false; break;
      }
      if (partials) write_block_partials<kPacked>(d.get(0), d.get(1), d.get(2), slot, sh.sm);
    }
    // The next pass may read this pass's stores with bulk copies (async proxy).
    if (STAGED) fence_proxy_async();
    if (!g.sync()) {
      if (threadIdx.x == 0) { C.status = PPCG_ERR_TIMEOUT; C.state = S_DONE; }
      break;
    }
    if (partials) {
      if constexpr (G::kCluster) cluster_reduce(sh.part[C.parity], C.red);
      else group_reduce(S.part + (size_t)C.parity * P * 4, P, C.red);
      if (threadIdx.x == 0) C.parity ^= 1;
    }
  }
  if constexpr (G::kCluster) {
    // other CTAs may still read this CTA's partials; the next system (or the exit) waits
    __syncthreads();
    cluster_barrier();
  }
  if (threadIdx.x == 0 && g.rank() == 0) {
    C.t_end = globaltimer();
    *S.ctl = C;
    __threadfence();
  }
}

template <int THREADS, int MINB, bool STAGED, bool BOX = false, int CM = kColA, bool PF = false>
__global__ void __launch_bounds__(THREADS, MINB) k_grid(const SysDesc* d, int budget) {
  __shared__ SharedT<kSmGrid> sh;
  __shared__ uint64_t bars[2 * (THREADS / 32)];
  extern __shared__ __align__(128) unsigned char stage_mem[];
  unsigned phases = 0;
  if (STAGED) {
    if ((threadIdx.x & 31) == 0) {
      mbar_init(bars + 2 * (threadIdx.x >> 5), 1);
      mbar_init(bars + 2 * (threadIdx.x >> 5) + 1, 1);
      mbar_init_fence();
    }
    __syncthreads();
  }
  GridGroup g{d->bar, d->err, (long long)d->spin_limit_ns, 0u};
  run_system<STAGED, BOX, CM, PF>(g, d, budget, sh, stage_mem, bars, phases);
}

// Launch shapes of the grid path: (threads per CTA, minimum CTAs per SM for the register
// budget, bulk-copy staging).  Index 0 is the default (fastest measured on the 256^3
// stencil); the others trade registers, resident warps and staging.  From kFirstBoxShape on:
// the kernels of matrix-free box-stencil plans; last, the default shape reading the column
// dictionary (plans whose matrix has one) and the default shape forming columns from the
// offset pattern (plans whose matrix has one).
struct GridShape {
  void (*fn)(const SysDesc*, int);
  int threads;
  int smem;     // dynamic shared memory (staging buffers)
};
const GridShape kGridShapes[] = {
    {k_grid<512, 2, false>, 512, 0}, {k_grid<256, 4, false>, 256, 0}, {k_grid<256, 3, false>, 256, 0},
    {k_grid<512, 1, false>, 512, 0}, {k_grid<384, 2, false>, 384, 0}, {k_grid<128, 6, false>, 128, 0},
    {k_grid<512, 1, true>, 512, 16 * kWarpStageBytes}, {k_grid<256, 2, true>, 256, 8 * kWarpStageBytes},
    {k_grid<384, 1, true>, 384, 12 * kWarpStageBytes},
    {k_grid<512, 2, false, true>, 512, 0}, {k_grid<256, 4, false, true>, 256, 0},
    {k_grid<1024, 1, false, true>, 1024, 0},
    {k_grid<512, 2, false, false, kColDict>, 512, 0},
    {k_grid<512, 2, false, false, kColPat>, 512, 0},
    // The FP32 forms' defaults: 20 warps per CTA at 48 registers (more spilling, more
    // warps in flight for the latency-bound FP32 passes: 256^3 stencil FP32_RU 2.6% and
    // 4M-point graph 6% faster than at 512 threads, where FP64 was 1-4% slower).
    {k_grid<640, 2, false>, 640, 0},
    {k_grid<640, 2, false, false, kColDict>, 640, 0},
    {k_grid<640, 2, false, false, kColPat>, 640, 0},
    // The offset-pattern default with the own-entry prefetch: FP64 systems whose vectors
    // exceed half the L2 (the prefetch code in the other kernel made small solves up to 7%
    // slower even when skipped).
    {k_grid<512, 2, false, false, kColPat, true>, 512, 0},
};
constexpr int kNumGridShapes = (int)(sizeof(kGridShapes) / sizeof(kGridShapes[0]));
constexpr int kFirstBoxShape = 9;
constexpr int kDictShape = 12;   // the default shape with the column dictionary
constexpr int kPatShape = 13;    // the default shape with the offset pattern
constexpr int kF32Shape = 14;    // the FP32 defaults: stored columns, dictionary, pattern
constexpr int kPatPfShape = 17;  // the offset-pattern default with the own-entry prefetch
static_assert(kPatPfShape + 1 == kNumGridShapes, "the prefetching pattern kernel is the last shape");

// Cluster path.  Static schedule (next == nullptr): cluster c runs list[list_ptr[c] ..
// list_ptr[c + 1]).  Dynamic schedule: every cluster takes the next entry of list (ordered
// longest first) from the counter *next until m entries are taken -- list scheduling, which
// absorbs the errors of any cost estimate.  A system's result does not depend on the
// cluster that runs it, only on the launch's cluster size (every system of a launch has
// the same one, fixed by its handle's plan).  Systems with an offset pattern run the
// pattern form of the passes (no column bytes), the others read their 4-byte columns.
__global__ void __launch_bounds__(kClusterThreads, 4) k_cluster(const SysDesc* descs, const int32_t* list,
                                                             const int32_t* list_ptr, int budget,
                                                             int32_t* next, int32_t m) {
  __shared__ SharedT<kSmCluster> sh;
  __shared__ int32_t sh_take;
  ClusterGroup g;
  unsigned cid;
  unsigned phases = 0;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
  auto run = [&](const SysDesc* d) {
    if (d->A.pat_k > 0) run_system<false, false, kColPat>(g, d, budget, sh, nullptr, nullptr, phases);
    else run_system<false>(g, d, budget, sh, nullptr, nullptr, phases);
  };
  if (!next) {
    for (int k = list_ptr[cid]; k < list_ptr[cid + 1]; k++) run(descs + list[k]);
    return;
  }
  const uint32_t rank = cluster_rank();
  for (;;) {
    if (rank == 0 && threadIdx.x == 0) sh_take = atomicAdd(next, 1);
    __syncthreads();
    cluster_barrier();   // rank 0's entry is visible to the cluster
    int32_t k;
    {
      uint32_t remote;
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_addr(&sh_take)), "r"(0u));
      asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(k) : "r"(remote));
    }
    __syncthreads();
    cluster_barrier();   // everyone has read it before rank 0 takes the next one
    if (k >= m) break;
    run(descs + list[k]);
  }
}

// ---------------------------------------------------------- on-chip small systems --
// A system whose vectors and matrix fit in the shared memory of one cluster of NC = 8 or 16
// CTAs (the launch's cluster size) runs entirely on chip: chunk c lives in CTA c % NC as
// local chunk c / NC (its FP64 vector tile and its SELL slots), gathers of other CTAs' rows
// are distributed-shared-memory loads, and
// the block partials are exchanged through shared memory as well.  No pass touches HBM or
// L2 except for b and the diagonal (setup, true residual, replacement).  The same
// control() drives it, so the iteration, its stopping rules, restarts and replacements are
// those of the other paths; the vector tiles are loaded at launch and written back at exit,
// so a solve can stop at an iteration budget and resume in a later launch.

// Eight warps work on the local chunks; a ninth (kOnchipCtl) owns none: it reduces the
// cluster's partials and runs the control step while the others compute, for the iteration
// that follows, the product of their first chunk (see k_onchip).
constexpr int kOnchipWork = 8, kOnchipCtl = kOnchipWork, kOnchipThreads = (kOnchipWork + 1) * 32;


// Gather of one slot of the distributed vector tiles: row j is lane j % 32 of chunk j / 32,
// held by CTA (j / 32) % NC as its local chunk (j / 32) / NC (NC = 1 << lg).
struct GatherDS {
  uint32_t tile;   // shared-memory address of the tile array (the same in every CTA)
  int slot;
  uint32_t lg;     // log2 of the cluster size
  __device__ __forceinline__ double operator()(int32_t j) const {
    const uint32_t cj = (uint32_t)j >> 5;
    const uint32_t off = (((cj >> lg) * (uint32_t)kNS64 + (uint32_t)slot) * kChunk + ((uint32_t)j & 31u)) * 8u;
    return ld_dsmem(tile + off, cj & ((1u << lg) - 1u));
  }
};

// acc + sum_k val[k] x(col[k]) (* dsc[col] when SCALE) over a row's slots in shared memory,
// in slot order (the order of row_dot).
template <bool SCALE, class G>
__device__ __forceinline__ double row_dot_sm(const int32_t* col, const double* val, const G& x,
                                             const double* __restrict__ dsc, int base, int len, double acc) {
  int j = 0;
  for (; j + 8 <= len; j += 8) {
    int32_t c[8];
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; k++) { c[k] = col[base + (j + k) * kChunk]; a[k] = val[base + (j + k) * kChunk]; }
#pragma unroll
    for (int k = 0; k < 8; k++) {
      double xv = x(c[k]);
      if (SCALE) xv = __ldg(dsc + c[k]) * xv;
      acc = fma(a[k], xv, acc);
    }
  }
  for (; j < len; j++) {
    const int32_t c = col[base + j * kChunk];
    double xv = x(c);
    if (SCALE) xv = __ldg(dsc + c) * xv;
    acc = fma(val[base + j * kChunk], xv, acc);
  }
  return acc;
}

struct OnchipSh {
  SysDesc S;
  Ctl C;
  double sm[3 * 32 * (kOnchipThreads / 32)];
  double part[2][4];     // this CTA's block partials, read by every CTA of the cluster
};

// Per-CTA view of the on-chip system.
struct Onchip {
  double* tile;          // [nloc][kNS64][32]
  double* val;           // this CTA's SELL slots (chunk after chunk)
  int32_t* col;
  int32_t* lptr;         // [nloc + 1] slot offset of each local chunk
  uint32_t tile_addr;
  int32_t nloc, rank, nchunks, n;
  int32_t nc, lg;        // cluster size and its log2
};

// Local chunks of this warp: lc = warp, warp + 8, ...; the control warp takes none.
#define FOR_LOCAL(O) \
  for (int32_t lc = (int32_t)(threadIdx.x >> 5); lc < (O).nloc && (threadIdx.x >> 5) < kOnchipWork; lc += kOnchipWork)

// The product n = Ahat w of local chunk lc, w in slot ws, for its rows (the first part of
// P_ITER; the same FMA sequence).
__device__ __forceinline__ double onchip_product(const Onchip& O, int32_t lc, int ws) {
  const int lane = threadIdx.x & 31;
  const int32_t c = lc * O.nc + O.rank;
  const bool in = c * kChunk + lane < O.n;
  const double* t = O.tile + (int64_t)lc * kNS64 * kChunk + lane;
  const int base = O.lptr[lc] + lane, len = (O.lptr[lc + 1] - O.lptr[lc]) / kChunk;
  const GatherDS gw{O.tile_addr, ws, (uint32_t)O.lg};
  return row_dot_sm<false>(O.col, O.val, gw, nullptr, base, len, in ? t[ws * kChunk] : 0.0);
}

// Products of a warp's first local chunks, formed ahead (see k_onchip): at most kOnchipSpec
// chunks, and beyond the first only while their slots add up to kOnchipSpecSlots -- about
// what fits in the control step's time.  4 chunks of a 3-D 24^3 stencil (6 slots each):
// solve 1289 -> 1110 us; 2 chunks of an 8k-point graph (~20 slots each) made it 2.7% slower.
constexpr int kOnchipSpec = 4, kOnchipSpecSlots = 24;
struct OnchipSpec {
  int n;                 // chunks formed
  double v[kOnchipSpec];
  __device__ __forceinline__ double get(int i) const {   // i < kOnchipSpec, register-resident
    double r = v[0];
#pragma unroll
    for (int k = 1; k < kOnchipSpec; k++) r = i == k ? v[k] : r;
    return r;
  }
};

// One on-chip pass; returns whether it produced partials.  spec: the products of this warp's
// first local chunks for this P_ITER, computed ahead (see k_onchip).
__device__ bool onchip_pass(const SysDesc& S, const Ctl& C, const Onchip& O, Dots<double>& d, bool paper,
                            bool spec_ok = false, const OnchipSpec* spec = nullptr) {
  const int lane = threadIdx.x & 31;
  const DevMatrix& A = S.A;
  switch (C.pass) {
    case P_SETUP1:
    case P_TRUE:
    case P_GAP:
    case P_RR1: {
      // r = b - A x (SCALE); setup1: u = M^-1 r, partials (b,b) (r,r); true: partial (r,r) only;
      // gap: partials ((b - A x) - r)^2, r^2; rr1: u = M^-1 r, s = A p, q = M^-1 s.
      const bool x_zero = C.pass == P_SETUP1 && S.x_zero != 0 && !C.fallback;
      const bool rr = C.pass == P_RR1, p_zero = rr && (C.iter == 0 || C.restart);
      const GatherDS gx{O.tile_addr, V_X, (uint32_t)O.lg}, gp{O.tile_addr, V_P, (uint32_t)O.lg};
      FOR_LOCAL(O) {
        const int32_t c = lc * O.nc + O.rank;
        if (c >= O.nchunks) continue;
        const int32_t row = c * kChunk + lane;
        const bool in = row < O.n;
        double* t = O.tile + (int64_t)lc * kNS64 * kChunk + lane;
        const int base = O.lptr[lc] + lane, len = (O.lptr[lc + 1] - O.lptr[lc]) / kChunk;
        double ax = 0.0, ap = 0.0, bi = 0.0, di = 0.0;
        if (in) {
          bi = __ldg(S.b + row);
          di = __ldg(A.diag + row);
          if (!x_zero) ax = di * t[V_X * kChunk];
          if (rr && !p_zero) ap = di * t[V_P * kChunk];
        }
        if (!x_zero) ax = row_dot_sm<true>(O.col, O.val, gx, A.diag, base, len, ax);
        if (rr && !p_zero) ap = row_dot_sm<true>(O.col, O.val, gp, A.diag, base, len, ap);
        if (in) {
          const double ri = bi - ax;
          if (C.pass == P_TRUE) { d.add(0, ri, ri); continue; }
          if (C.pass == P_GAP) {
            const double rr_i = t[V_R * kChunk], gi = ri - rr_i;
            d.add(0, gi, gi);
            d.add(1, rr_i, rr_i);
            continue;
          }
          const double id = t[V_INVD * kChunk];
          t[V_R * kChunk] = ri;
          t[V_U * kChunk] = id * ri;
          if (rr) {
            t[V_S * kChunk] = ap;
            t[V_Q * kChunk] = id * ap;
          } else {
            d.add(0, bi, bi);
            d.add(1, ri, ri);
          }
        }
      }
      return !rr;
    }
    case P_SETUP2:
    case P_RR2: {
      // w = Ahat r (= A u); rr2 also z = Ahat s (= A q); partials (r,u) (w,u) norm.
      const bool rr = C.pass == P_RR2;
      const int wcs = rr && (C.iter & 1) ? V_WB : V_WA;
      const GatherDS gr{O.tile_addr, V_R, (uint32_t)O.lg}, gs{O.tile_addr, V_S, (uint32_t)O.lg};
      FOR_LOCAL(O) {
        const int32_t c = lc * O.nc + O.rank;
        if (c >= O.nchunks) continue;
        const bool in = c * kChunk + lane < O.n;
        double* t = O.tile + (int64_t)lc * kNS64 * kChunk + lane;
        const int base = O.lptr[lc] + lane, len = (O.lptr[lc + 1] - O.lptr[lc]) / kChunk;
        double ri = 0.0, ui = 0.0, si = 0.0;
        if (in) { ri = t[V_R * kChunk]; ui = t[V_U * kChunk]; if (rr) si = t[V_S * kChunk]; }
        const double wi = row_dot_sm<false>(O.col, O.val, gr, nullptr, base, len, ri);
        double zi = 0.0;
        if (rr) zi = row_dot_sm<false>(O.col, O.val, gs, nullptr, base, len, si);
        if (in) {
          t[wcs * kChunk] = wi;
          if (rr) t[V_Z * kChunk] = zi;
          d.add(0, ri, ui);
          d.add(1, wi, ui);
          if (paper) d.add(2, ui, ui); else d.add(2, ri, ri);
        }
      }
      return true;
    }
    case P_ITER: {
      const bool first = C.first != 0, with_rr = C.want_rr != 0;
      const double alpha = C.alpha, beta = C.beta;
      const int wcs = (C.iter & 1) ? V_WB : V_WA;
      const int wns = (C.iter & 1) ? V_WA : V_WB;
      const GatherDS gw{O.tile_addr, wcs, (uint32_t)O.lg};
      FOR_LOCAL(O) {
        const int32_t c = lc * O.nc + O.rank;
        if (c >= O.nchunks) continue;
        const bool in = c * kChunk + lane < O.n;
        double* t = O.tile + (int64_t)lc * kNS64 * kChunk + lane;
        const int base = O.lptr[lc] + lane, len = (O.lptr[lc + 1] - O.lptr[lc]) / kChunk;
        double wi = 0.0;
        if (in) wi = t[wcs * kChunk];
        // n_i = (A M^-1 w)_i = w_i + sum_{j != i} ahat_ij w_j
        const int si = (lc - (int32_t)(threadIdx.x >> 5)) / kOnchipWork;   // this warp's i-th chunk
        const double ni = spec_ok && si < spec->n ? spec->get(si)
                                                      : row_dot_sm<false>(O.col, O.val, gw, nullptr, base, len, wi);
        if (in) {
          const double id = t[V_INVD * kChunk], ui = t[V_U * kChunk];
          const double mi = id * wi;
          const double zi = first ? ni : fma(beta, t[V_Z * kChunk], ni);
          const double qi = first ? mi : fma(beta, t[V_Q * kChunk], mi);
          const double si = first ? wi : fma(beta, t[V_S * kChunk], wi);
          const double pi = first ? ui : fma(beta, t[V_P * kChunk], ui);
          const double xi = fma(alpha, pi, t[V_X * kChunk]);
          const double ri = fma(-alpha, si, t[V_R * kChunk]);
          const double un = fma(-alpha, qi, ui);
          const double wnn = fma(-alpha, zi, wi);
          t[V_Z * kChunk] = zi;
          t[V_Q * kChunk] = qi;
          t[V_S * kChunk] = si;
          t[V_P * kChunk] = pi;
          t[V_X * kChunk] = xi;
          t[V_R * kChunk] = ri;
          t[V_U * kChunk] = un;
          t[wns * kChunk] = wnn;
          d.add(0, ri, un);
          d.add(1, wnn, un);
          if (with_rr) { if (paper) d.add(2, un, un); else d.add(2, ri, ri); }
        }
      }
      return true;
    }
    case P_NORM: {
      FOR_LOCAL(O) {
        const int32_t c = lc * O.nc + O.rank;
        if (c >= O.nchunks || c * kChunk + lane >= O.n) continue;
        const double v = O.tile[((int64_t)lc * kNS64 + (paper ? V_U : V_R)) * kChunk + lane];
        d.add(2, v, v);
      }
      return true;
    }
    case P_ZERO_X: {
      FOR_LOCAL(O) {
        const int32_t c = lc * O.nc + O.rank;
        if (c < O.nchunks && c * kChunk + lane < O.n) O.tile[((int64_t)lc * kNS64 + V_X) * kChunk + lane] = 0.0;
      }
      return false;
    }
    default:
      return false;
  }
}

// Copy this CTA's chunks between the global vector block and the shared tiles.
__device__ void onchip_tiles(const SysDesc& S, const Onchip& O, bool to_smem) {
  const int64_t per = (int64_t)kNS64 * kChunk;
  for (int64_t k = threadIdx.x; k < (int64_t)O.nloc * per; k += blockDim.x) {
    const int64_t lc = k / per, e = k % per;
    const int64_t c = lc * O.nc + O.rank;
    if (c >= O.nchunks) continue;
    double* g = S.v64 + c * per + e;
    if (to_smem) O.tile[k] = __ldcg(g); else __stcg(g, O.tile[k]);
  }
}

__global__ void __launch_bounds__(kOnchipThreads, 1) k_onchip(const SysDesc* descs, const int32_t* list,
                                                              const int32_t* list_ptr, int budget_arg) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ OnchipSh sh;
  unsigned cid;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
  const uint32_t rank = cluster_rank();
  for (int item = list_ptr[cid]; item < list_ptr[cid + 1]; item++) {
    const SysDesc* Sg = descs + list[item];
    __syncthreads();
    if (threadIdx.x == 0) {
      sh.S = *Sg;
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(sh.S.ctl);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sh.C);
      for (int i = 0; i < (int)(sizeof(Ctl) / 8); i++) dst[i] = __ldcg(src + i);
      if (sh.C.t_start == 0) sh.C.t_start = globaltimer();
      sh.C.exit_now = 0;
    }
    __syncthreads();
    const SysDesc& S = sh.S;
    Ctl& C = sh.C;
    Onchip O;
    O.nchunks = (int32_t)S.A.nchunks;
    O.n = (int32_t)S.A.n;
    O.rank = (int32_t)rank;
    O.nc = (int32_t)cluster_nranks();
    O.lg = O.nc == 16 ? 4 : 3;
    O.nloc = (O.nchunks + O.nc - 1) / O.nc;
    O.tile = reinterpret_cast<double*>(dyn);
    O.val = O.tile + (int64_t)O.nloc * kNS64 * kChunk;
    O.col = reinterpret_cast<int32_t*>(O.val + S.onchip_slots);
    O.lptr = O.col + S.onchip_slots;
    O.tile_addr = smem_u32(O.tile);
    // stage: local slot offsets, then the matrix slots and the vector tiles
    if (threadIdx.x == 0) {
      int32_t off = 0;
      for (int32_t lc = 0; lc < O.nloc; lc++) {
        O.lptr[lc] = off;
        const int64_t c = (int64_t)lc * O.nc + rank;
        if (c < O.nchunks) off += (int32_t)(__ldg(S.A.cptr + c + 1) - __ldg(S.A.cptr + c));
      }
      O.lptr[O.nloc] = off;
    }
    __syncthreads();
    for (int32_t lc = (int32_t)(threadIdx.x >> 5); lc < O.nloc; lc += kOnchipThreads / 32) {
      const int64_t c = (int64_t)lc * O.nc + rank;
      if (c >= O.nchunks) continue;
      const int64_t g0 = __ldg(S.A.cptr + c);
      const int cnt = O.lptr[lc + 1] - O.lptr[lc];
      for (int k = threadIdx.x & 31; k < cnt; k += 32) {
        O.col[O.lptr[lc] + k] = __ldg(S.A.col + g0 + k);
        O.val[O.lptr[lc] + k] = __ldg(S.A.val + g0 + k);
      }
    }
    onchip_tiles(S, O, true);
    int budget = budget_arg;
    if (S.budget > 0) budget = S.budget;
    const int iter_end = budget > 0 && C.iter < 0x7fffffff - budget ? C.iter + budget : 0x7fffffff;
    const bool paper = S.norm == PPCG_NORM_PAPER_U_ABS;
    __syncthreads();
    cluster_barrier();   // every CTA's tiles are staged before anyone gathers
    // Speculative products: after a P_ITER pass, while warp kOnchipCtl reduces the partials
    // and runs the control step, each working warp forms the products its first
    // kOnchipSpec local chunks need in the next iteration (slot wns of the pass just done is
    // that iteration's w), in registers.
    // It is used when the control step indeed continues with P_ITER of that iteration;
    // nothing can have written the slot in between: the one pass another CTA may run
    // meanwhile is the one that control step chose (P_ITER, P_NORM, P_GAP, P_TRUE or P_RR1),
    // and none of them writes wns of the iteration before.
    const int warp = (int)(threadIdx.x >> 5);
    bool spec_ok = false;
    OnchipSpec spec;
    int spec_iter = -1;
    for (;;) {
      if (threadIdx.x == kOnchipCtl * 32) control(C, S, iter_end);
      __syncthreads();
      if (C.pass == P_NONE) break;
      const int pass = C.pass, iter = C.iter;
      Dots<double> d;
      const bool use = spec_ok && pass == P_ITER && iter == spec_iter;
      const bool partials = onchip_pass(S, C, O, d, paper, use, &spec);
      if (partials) {
        write_block_partials<true>(d.get(0), d.get(1), d.get(2), sh.part[C.parity], sh.sm);
      }
      __syncthreads();
      cluster_barrier();
      spec_ok = false;
      if (warp == kOnchipCtl) {
        if (partials) {
          // lane q < NC reads rank q's partials; a fixed shuffle tree sums them (deterministic)
          const int lane = threadIdx.x & 31;
          const uint32_t base = smem_u32(&sh.part[C.parity][0]);
          double s0 = 0.0, s1 = 0.0, s2 = 0.0;
          if (lane < O.nc) {
            s0 = ld_dsmem(base, lane);
            s1 = ld_dsmem(base + 8, lane);
            s2 = ld_dsmem(base + 16, lane);
          }
          for (int o = O.nc / 2; o > 0; o >>= 1) {
            s0 += __shfl_down_sync(kFull, s0, o);
            s1 += __shfl_down_sync(kFull, s1, o);
            s2 += __shfl_down_sync(kFull, s2, o);
          }
          if (lane == 0) {
            C.red[0] = s0; C.red[1] = s1; C.red[2] = s2; C.red[3] = 0.0;
            C.parity ^= 1;
          }
        }
      } else if (pass == P_ITER) {
        spec.n = 0;
        int slots = 0;
#pragma unroll
        for (int i = 0; i < kOnchipSpec; i++) {
          const int32_t lc = warp + i * kOnchipWork;
          if (lc >= O.nloc || lc * O.nc + O.rank >= O.nchunks) break;
          slots += (O.lptr[lc + 1] - O.lptr[lc]) / kChunk;
          if (i > 0 && slots > kOnchipSpecSlots) break;
          spec.v[i] = onchip_product(O, lc, (iter & 1) ? V_WA : V_WB);
          spec.n = i + 1;
        }
        spec_ok = true;
        spec_iter = iter + 1;
      }
    }
    cluster_barrier();   // no CTA reads another's shared memory after this point
    onchip_tiles(S, O, false);
    if (threadIdx.x == 0 && rank == 0) {
      C.t_end = globaltimer();
      *S.ctl = C;
      __threadfence();
    }
    __syncthreads();
  }
}

// Failure-detection self test: the grid barrier with one rank that never arrives.  Every
// other CTA must give up after limit_ns and report PPCG_ERR_TIMEOUT instead of hanging.
__global__ void k_barrier_selftest(unsigned* bar, int32_t* err, int32_t* out, int drop_rank,
                                   long long limit_ns) {
  GridGroup g{bar, err, limit_ns, 0u};
  if ((int)blockIdx.x == drop_rank) return;
  bool ok = g.sync();
  if (threadIdx.x == 0) out[blockIdx.x] = ok ? 1 : 0;
}

}  // namespace

int grid_shape_count() { return kFirstBoxShape; }
int grid_box_shape_first() { return kFirstBoxShape; }
int grid_box_shape_count() { return kDictShape - kFirstBoxShape; }
int grid_default_shape(int cols, bool fp32, bool streaming) {
  const int c = cols == PPCG_COLS_PATTERN ? 2 : cols == PPCG_COLS_DICT ? 1 : 0;
  return fp32 ? kF32Shape + c : c == 2 ? (streaming ? kPatPfShape : kPatShape) : c == 1 ? kDictShape : 0;
}
int grid_shape_cols(int shape) {
  if (shape == kPatShape || shape == kPatPfShape || shape == kF32Shape + 2) return PPCG_COLS_PATTERN;
  if (shape == kDictShape || shape == kF32Shape + 1) return PPCG_COLS_DICT;
  return PPCG_COLS_SELL;
}
int grid_threads(int shape) { return kGridShapes[shape].threads; }

cudaError_t ensure_smem_attr(const void* fn, size_t bytes);

static void set_smem_attr(const GridShape& gs) {
  if (gs.smem > 0 && ensure_smem_attr((const void*)gs.fn, (size_t)gs.smem) != cudaSuccess) cudaGetLastError();
}

int grid_blocks_for_device(int device, int shape) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const GridShape& gs = kGridShapes[shape];
  set_smem_attr(gs);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gs.fn, gs.threads, gs.smem);
  if (per < 1) per = 1;
  return sms * per;
}

// Cluster sizes above the portable 8 need the kernel's opt-in (once per device and kernel).
static cudaError_t allow_large_clusters(const void* fn) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, cudaError_t> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find({dev, fn});
  if (it != done.end()) return it->second;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) cudaGetLastError();
  done[{dev, fn}] = e;
  return e;
}

int max_active_clusters(int device, int cs) {
  (void)device;
  if (cs > 8 && allow_large_clusters((const void*)k_cluster) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs * 64);
  cfg.blockDim = dim3(kClusterThreads);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)k_cluster, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_grid(const SysDesc* d_desc, int shape, int grid, int budget, cudaStream_t st) {
  void* args[] = {(void*)&d_desc, (void*)&budget};
  const GridShape& gs = kGridShapes[shape];
  return cudaLaunchCooperativeKernel((void*)gs.fn, dim3(grid), dim3(gs.threads), args, gs.smem, st);
}

// Raise a kernel's dynamic shared memory limit to at least `bytes` on the current device
// (the attribute is per device; callers may run on several devices and host threads).
cudaError_t ensure_smem_attr(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = done[{dev, fn}];
  if (bytes <= have) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) have = bytes;
  return e;
}

cudaError_t launch_clusters(const SysDesc* d_descs, const int32_t* d_list, const int32_t* d_list_ptr,
                            int nclusters, int budget, cudaStream_t st, bool spread, int32_t* d_next, int32_t m,
                            int cs) {
  if (cs != 2 && cs != 4 && cs != 8 && cs != 16) return cudaErrorInvalidValue;
  if (cs > 8) {
    cudaError_t e = allow_large_clusters((const void*)k_cluster);
    if (e != cudaSuccess) return e;
  }
  // spread: request enough dynamic shared memory that no two CTAs share an SM, so a lone
  // cluster gets the FP64 pipes of cs SMs instead of being packed onto a few.
  const int spread_smem = 120 * 1024;
  if (spread && ensure_smem_attr((const void*)k_cluster, spread_smem) != cudaSuccess) cudaGetLastError();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs * nclusters);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = spread ? spread_smem : 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_cluster, d_descs, d_list, d_list_ptr, budget, d_next, m);
}

size_t onchip_smem_bytes(int64_t nchunks, int64_t slots, int nc) {
  const int64_t nloc = (nchunks + nc - 1) / nc;
  return (size_t)(nloc * kNS64 * kChunk * 8 + slots * 12 + (nloc + 1) * 4);
}

size_t onchip_smem_limit(int device) {
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  const size_t stat = sizeof(OnchipSh) + 1024;   // static shared memory and a reserve
  return optin > (int)stat ? (size_t)optin - stat : 0;
}

// The 16-CTA cluster is beyond the portable size: the kernel must opt in (once per device).
static cudaError_t allow_cluster16() { return allow_large_clusters((const void*)k_onchip); }

bool onchip_cluster_fits(int nc, size_t smem) {
  if (nc == 16 && allow_cluster16() != cudaSuccess) return false;
  if (ensure_smem_attr((const void*)k_onchip, smem) != cudaSuccess) { cudaGetLastError(); return false; }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(kOnchipThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = nc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (void*)k_onchip, &cfg) != cudaSuccess) { cudaGetLastError(); return false; }
  return n >= 1;
}

cudaError_t launch_onchip(const SysDesc* d_descs, const int32_t* d_list, const int32_t* d_list_ptr,
                          int nclusters, int budget, size_t smem, int nc, cudaStream_t st) {
  if (nc != 8 && nc != 16) return cudaErrorInvalidValue;
  if (nc == 16) {
    cudaError_t e = allow_cluster16();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = ensure_smem_attr((const void*)k_onchip, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc * nclusters);
  cfg.blockDim = dim3(kOnchipThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = nc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_onchip, d_descs, d_list, d_list_ptr, budget);
}

cudaError_t launch_barrier_selftest(unsigned* bar, int32_t* err, int32_t* out, int grid, int drop_rank,
                                    int64_t limit_ns, cudaStream_t st) {
  long long lim = (long long)limit_ns;
  void* args[] = {(void*)&bar, (void*)&err, (void*)&out, (void*)&drop_rank, (void*)&lim};
  return cudaLaunchCooperativeKernel((void*)k_barrier_selftest, dim3(grid), dim3(64), args, 0, st);
}

}  // namespace ppcg
