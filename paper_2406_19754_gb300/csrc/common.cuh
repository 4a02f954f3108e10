// Internal declarations shared by the translation units of the GPU library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <functional>
#include <vector>

#include "amg.h"

namespace amg {

// ------------------------------------------------------------------ errors

struct Status {
  int code = AMG_OK;
};

#define AMG_CUDA_TRY(...)                                    \
  do {                                                       \
    cudaError_t _e = (__VA_ARGS__);                          \
    if (_e != cudaSuccess) {                                 \
      amg::note_cuda_error(_e, #__VA_ARGS__, __FILE__, __LINE__); \
      return _e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA; \
    }                                                        \
  } while (0)

#define AMG_TRY(...)         \
  do {                       \
    int _s = (__VA_ARGS__);  \
    if (_s < 0) return _s;   \
  } while (0)

#define AMG_LAUNCH_CHECK() AMG_CUDA_TRY(cudaGetLastError())

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// ------------------------------------------------------------------ memory

// Device allocation used by every internal buffer (a failing allocation
// turns into AMG_ERR_OOM).  Allocations are tracked by their owner.
struct Arena {
  std::vector<void*> blocks;
  int alloc(void** p, size_t bytes);
  template <typename T>
  int alloc_n(T** p, int64_t n) {
    return alloc((void**)p, sizeof(T) * (size_t)(n > 0 ? n : 1));
  }
  void release(void* p);
  void release_all();
};

// ------------------------------------------------------------------ SELL

// Sliced ELLPACK (Sec. 2.2, "Hacked ELLPACK"): rows in slices of C rows,
// each slice an ELLPACK block of width = its longest row, stored column
// major (entry k of row r of slice s at sliceptr[s] + k * C + r).  Padding
// entries carry val = 0 and a valid column (the row itself).
// Batched systems: every system starts a new slice, so slice s covers rows
// [row0[s], row0[s+1]) (at most C rows) and belongs to system sys[s].
// Without systems row0/sys are null and slice s covers rows [s*C, s*C + C).
struct Sell {
  int64_t n = 0, nslices = 0, nnz_pad = 0;
  int C = 32, tpr = 1;
  int wmax = 0;  // widest slice (ELL columns)
  int64_t* sliceptr = nullptr;
  int32_t* col = nullptr;
  double* v64 = nullptr;
  float* v32 = nullptr;
  __nv_bfloat16* v16 = nullptr;
  int64_t* row0 = nullptr;  // nslices + 1, or null
  int32_t* sys = nullptr;   // nslices, or null
  // Compressed columns (null when some slice does not fit): ELL column k of
  // slice s (the C slots sliceptr[s] + k*C + [0, C)) has base
  // kbase[sliceptr[s]/C + k], and slot e holds column kbase[..] + d16[e].
  // The kernels stream d16 (2 bytes a slot) instead of col (4 bytes).
  uint16_t* d16 = nullptr;
  int32_t* kbase = nullptr;
};

template <typename V>
struct SellView {
  int64_t n, nslices;
  // Warp row-groups of the one-warp-per-group kernels (sellk.cuh): 32/tpr
  // consecutive rows each; the slices themselves when the slice height C is
  // 32/tpr, more or fewer groups than slices otherwise (C in {4, ..., 64}).
  int64_t ngroups;
  int C;
  const int64_t* sliceptr;
  const int32_t* col;
  const V* val;
  const int64_t* row0;
  const int32_t* sys;
  const uint16_t* d16;   // compressed columns, or null
  const int32_t* kbase;
  const int* act;        // batched PCG: per-system "still iterating" flags, or null
  // false for a slice of a system whose solve has stopped (its results are
  // not used), so the kernels skip it
  __device__ __forceinline__ bool live(int64_t s) const { return !act || act[sys[s]]; }
  // first row of slice s and one past its last row
  __device__ __forceinline__ int64_t rbeg(int64_t s, int C) const {
    return row0 ? __ldg(row0 + s) : s * C;
  }
  __device__ __forceinline__ int64_t rend(int64_t s, int C) const {
    if (row0) return __ldg(row0 + s + 1);
    const int64_t e = (s + 1) * C;
    return e < n ? e : n;
  }
};

// Value storage of a level in the V-cycle.
enum { VAL_F64 = 0, VAL_F32 = 1, VAL_BF16 = 2 };

struct Level {
  int64_t n = 0, nnz = 0;
  // FP64 CSR (levels >= 1; level 0 belongs to the caller)
  int64_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  Sell A;
  // V-cycle operators (levels above the coarsest):
  //   Ah = A S  (a_ij s_j; same slices and columns as A, own values)
  //   AP = A P  (row i, column J: sum of a_ij over agg(j) = J; own slices)
  double* ah64 = nullptr;
  float* ah32 = nullptr;
  __nv_bfloat16* ah16 = nullptr;
  Sell AP;
  int64_t ap_nnz = 0;
  int vstore = VAL_F64;
  double* d = nullptr;     // l1 row sums
  double* dinv = nullptr;  // 1 / d
  double* s64 = nullptr;   // smoother scale s_i = omega_i * (1 / d_i)
  float* s32 = nullptr;
  int32_t* agg = nullptr;      // row -> aggregate on level l+1
  int32_t* members = nullptr;  // nc x stride, ascending, -1 padded
  int stride = 0;
  int64_t nc = 0;
  // V-cycle work vectors of the V-cycle compute type
  void* b = nullptr;
  void* x = nullptr;
  void* r = nullptr;
  // smoother sweeps on this level (options smooth_sweeps / variable_cycle);
  // with nu > 1: a second residual buffer and the pre-smoothed x
  int64_t nu = 1;
  void* r2 = nullptr;
  void* xp = nullptr;
  // batched systems: first row of each system on this level (nsys + 1, host)
  std::vector<int64_t> sys_off;
  // smoothed prolongator (option smooth_prolongator, Sec. 2.3): P = (I - w
  // D^-1 A) P_hat (n x nc CSR, kept for export, and sliced ELL with A's
  // slices), its transpose R = P^T as sliced ELL (restriction), and AP above
  // then holds A P.  The CSRs of R and A P live only until setup has made
  // their sliced-ELL copies.
  double wp = 0.0;
  int64_t* p_rp = nullptr;
  int32_t* p_ci = nullptr;
  double* p_v = nullptr;
  int64_t p_nnz = 0;
  int64_t* t_rp = nullptr;
  int32_t* t_ci = nullptr;
  double* t_v = nullptr;
  int64_t* q_rp = nullptr;
  int32_t* q_ci = nullptr;
  double* q_v = nullptr;
  int64_t q_nnz = 0;
  Sell P, R;
};

// Batched PCG state (pcg_solve_batch): per-system scalars and per-slice
// partial sums over the level-0 slices, which never straddle two systems.
// Level-0 slices of each system are grouped into chunks of at most
// BATCH_CHUNK consecutive slices; a warp walks whole chunks, keeps its dot
// sums per thread over a chunk's slices and writes one pair of partials per
// chunk (one warp reduction per chunk, none inside the slice loop).
constexpr int BATCH_CHUNK = 16;

struct Batch {
  int nsys = 0;
  int64_t nslices = 0;
  int64_t* slice_off = nullptr;  // device, nsys + 1: slices of system k
  int64_t nchunks = 0;
  int64_t* chunk_off = nullptr;  // device, nchunks + 1: first slice of chunk c
  int64_t* sys_chunk = nullptr;  // device, nsys + 1: first chunk of system k
  double* part = nullptr;        // device, 2 * nchunks: per-chunk partial sums
  struct Scal* sc = nullptr;     // device, nsys
  struct Scal* sc_host = nullptr;  // pinned, nsys
  int* active = nullptr;         // device, nsys: copy of each system's active flag
  int* nactive = nullptr;        // device counter
  int* loop_ctl = nullptr;       // device: iteration count and cap of the loop graph
};

struct Scal {
  double bb, rr, rz, pq, zq, alpha, beta, tr;
  int status, active, iters, pq_fail;
};

// Device-resident PCG scalars.
struct PcgScalars {
  double bb, rr, rz, pq, zq, alpha, beta;
  int status;
  int beta_form;
  int pq_fail;
  // device-side stopping test of the graph-resident loop (pcg.cu)
  double tol;
  int maxit;
  int iter;
  // 1 while x += alpha p of the last update is still to be applied (pcg.cu)
  int x_pending;
};

// Coarsest blocks up to this many rows are factored and solved by one CUDA
// block each; larger ones use kernels spread over the whole GPU.
constexpr int64_t COARSE_SMALL = 1024;

// Diagonal block of coarsest row i: b with brow[b] <= i < brow[b+1].
__device__ __forceinline__ int coarse_block(const int64_t* brow, int nblk, int64_t i) {
  int lo = 0, hi = nblk;
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (brow[mid] <= i)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Deterministic grid reduction scratch: per-block partials + ticket.
struct Reduce {
  double* partials = nullptr;  // [max_blocks * 4]
  unsigned* ticket = nullptr;
  int max_blocks = 0;
};

}  // namespace amg

struct amg_handle {
  amg_options opt;
  int device = 0;
  int num_sms = 0;
  amg::Arena arena;
  std::vector<amg::Level> L;
  int64_t nco = 0;
  // coarsest level: block diagonal (one block per batched system, else one);
  // block b has rows [brow[b], brow[b+1]) and its L^-1 and L^-T (row-major,
  // dense) start at bmat[b] in Linv / LinvT
  int nblk = 1;
  std::vector<int64_t> cblk_row;
  int64_t* d_brow = nullptr;
  int64_t* d_bmat = nullptr;
  double* Linv = nullptr;
  double* LinvT = nullptr;
  double* coarse_y = nullptr;  // nco: intermediate of the large-block coarse solve
  double* cpcg = nullptr;      // 5 * nco: x, r, z, p, q of the PCG coarsest solve
  // PCG workspace
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
  float* r32 = nullptr;  // FP32 copy of r for an FP32 V-cycle (else null)
  amg::PcgScalars* sc = nullptr;
  amg::PcgScalars* sc_host = nullptr;  // pinned
  amg::Reduce red;
  int* dev_status = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  const double* graph_b = nullptr;
  double* graph_x = nullptr;
  int graph_beta = -2;
  int graph_defer = -1;
  // the whole PCG loop as one graph (device-side stopping test in a
  // conditional while node); loop_state 0 untried, 1 built, -1 unavailable
  cudaGraphExec_t loop = nullptr;
  double* loop_x = nullptr;
  int loop_beta = -2;
  int loop_state = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // batched systems (amg_setup_batch); nsys == 1 otherwise
  bool batched = false;
  int nsys = 1;
  std::vector<int64_t> sys_off0;  // first row of each system (nsys + 1)
  amg::Batch batch;
  cudaGraphExec_t bgraph = nullptr;
  double* bgraph_x = nullptr;
  int bgraph_beta = -2;
  double bgraph_tol = -1.0;
  int bgraph_maxit = -1;
  cudaGraphExec_t bloop = nullptr;  // batched loop graph (device-side stop)
  double* bloop_x = nullptr;
  int bloop_beta = -2;
  double bloop_tol = -1.0;
  int bloop_maxit = -1;
  int bloop_state = 0;
  void* multi = nullptr;  // multi-RHS workspace (multi.cu)
  void* tg = nullptr;     // two-grid loss workspace and inner solver (twogrid.cu)
  // persistent small-level launch (tail.cu): grid-barrier word, sticky
  // failure flag, and the largest co-resident grid (0: not available)
  unsigned* tail_bar = nullptr;
  int* tail_fail = nullptr;
  // sticky flag of the streaming kernels (ring.cuh): set when a bounded wait
  // for a bulk copy gave up; later launches return at once until it is read
  int* wait_fail = nullptr;
  int tail_grid = 0;
  int tail_debug = 0;  // amg_debug_tail_timeout
  unsigned long long pattern = 0;  // fingerprint of the level-0 sparsity (value updates)
};

namespace amg {

// Stages per warp of the shared-memory ring streams (option stream_ring:
// 0 off, 1 the default count, 2..4 that many); 0 means the default.
inline int ring_stages(const amg_handle* H) {
  return H->opt.stream_ring >= 2 ? H->opt.stream_ring : 0;
}

// ------------------------------------------------------------------ device helpers

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  // splitmix64 finaliser (Steele, Lea, Flood 2014)
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
  return __ldcs(p);
}
template <>
__device__ __forceinline__ __nv_bfloat16 ld_stream<__nv_bfloat16>(const __nv_bfloat16* p) {
  return *p;
}

__device__ __forceinline__ double to_f(double v, double) { return v; }
__device__ __forceinline__ float to_f(float v, float) { return v; }
__device__ __forceinline__ float to_f(double v, float) { return (float)v; }
__device__ __forceinline__ double to_f(float v, double) { return (double)v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v, float) { return __bfloat162float(v); }
__device__ __forceinline__ double to_f(__nv_bfloat16 v, double) {
  return (double)__bfloat162float(v);
}

// Conversions between binary64 and binary32 on the integer pipe, for kernels
// that convert every element of a blocked (N x K) vector.  GB300's FP64 pipe,
// which also executes the conversion instructions, retires about two lane
// operations per SM clock, so such a kernel is bound by it.  For a value in
// binary32's normal range the conversions are bit operations on the IEEE 754
// encodings (1 sign, 11 exponent bits biased by 1023 and 52 fraction bits;
// 1, 8 biased by 127, 23): rebias the exponent, keep the top 23 fraction
// bits, and round to nearest, ties to even, on the 29 dropped bits.  Zeros
// take the bit path too.  Any other input (NaN, infinity, subnormal or out of
// range: rare in the solver's vectors) clears `ok`, and the array forms below
// then convert the whole array in hardware.  There is no branch per element,
// so a caller's loads all issue before the first conversion.  The results are
// the hardware conversion's bits.
__device__ __forceinline__ float f64_to_f32_bits(double x, bool& ok) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  const uint32_t e = (hi >> 20) & 0x7FFu;
  const bool in = e - 897u < 254u;  // binary32 biased exponent e - 896 in 1..254
  uint32_t r = ((e - 896u) << 23) | (__funnelshift_l(lo, hi, 3) & 0x7FFFFFu);
  // carry out of the dropped bits: above half, or exactly half and r odd; a
  // carry out of the fraction steps the exponent (to infinity past 254)
  r += ((lo & 0x1FFFFFFFu) + 0x0FFFFFFFu + (r & 1u)) >> 29;
  ok = ok && (in || ((hi << 1) | lo) == 0u);
  return __uint_as_float((hi & 0x80000000u) | (in ? r : 0u));
}

// Exact: a normal binary32 value's exponent rebiased by 1023 - 127 = 896,
// its 23 fraction bits the top of the 52.
__device__ __forceinline__ double f32_to_f64_bits(float f, bool& ok) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t m = u & 0x7FFFFFFFu;
  const bool in = (m >> 23) - 1u < 254u;  // biased exponent 1..254
  ok = ok && (in || m == 0u);
  return __hiloint2double((int)((u & 0x80000000u) | (in ? (m >> 3) + (896u << 20) : 0u)),
                          (int)(in ? u << 29 : 0u));
}

// The hardware conversions of a whole array, out of line: inlined, the
// compiler predicates them into the caller, and predicated-off FP64-pipe
// instructions still take the pipe's cycles.
template <typename A, typename B, int N>
struct CvtArr {
  B v[N];
};
template <int N>
__device__ __noinline__ CvtArr<double, float, N> cvt_hw(CvtArr<double, double, N> a) {
  CvtArr<double, float, N> r;
#pragma unroll
  for (int q = 0; q < N; ++q) r.v[q] = __double2float_rn(a.v[q]);
  return r;
}
template <int N>
__device__ __noinline__ CvtArr<float, double, N> cvt_hw(CvtArr<float, float, N> a) {
  CvtArr<float, double, N> r;
#pragma unroll
  for (int q = 0; q < N; ++q) r.v[q] = (double)a.v[q];
  return r;
}

template <int N>
__device__ __forceinline__ void cvt_n(const double (&in)[N], float (&out)[N]) {
  bool ok = true;
#pragma unroll
  for (int q = 0; q < N; ++q) out[q] = f64_to_f32_bits(in[q], ok);
  if (!ok) {
    CvtArr<double, double, N> a;
#pragma unroll
    for (int q = 0; q < N; ++q) a.v[q] = in[q];
    const CvtArr<double, float, N> r = cvt_hw<N>(a);
#pragma unroll
    for (int q = 0; q < N; ++q) out[q] = r.v[q];
  }
}
template <int N>
__device__ __forceinline__ void cvt_n(const float (&in)[N], double (&out)[N]) {
  bool ok = true;
#pragma unroll
  for (int q = 0; q < N; ++q) out[q] = f32_to_f64_bits(in[q], ok);
  if (!ok) {
    CvtArr<float, float, N> a;
#pragma unroll
    for (int q = 0; q < N; ++q) a.v[q] = in[q];
    const CvtArr<float, double, N> r = cvt_hw<N>(a);
#pragma unroll
    for (int q = 0; q < N; ++q) out[q] = r.v[q];
  }
}
template <int N, typename T>
__device__ __forceinline__ void cvt_n(const T (&in)[N], T (&out)[N]) {
#pragma unroll
  for (int q = 0; q < N; ++q) out[q] = in[q];
}
template <int N>
__device__ __forceinline__ void cvt_n(const __nv_bfloat16 (&in)[N], float (&out)[N]) {
#pragma unroll
  for (int q = 0; q < N; ++q) out[q] = __bfloat162float(in[q]);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over a block; result valid in thread 0.  Fixed tree => deterministic.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][w] = v[k];
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < nw ? sh[k][lane] : 0.0;
      v[k] = warp_sum(t);
    }
  }
}

// Last block of a grid reduction: adds all block partials in block order
// (fixed tree) and runs `epi(total)` in thread 0.  Kept out of line so its
// registers do not count against the streaming loop of the calling kernel.
template <int NV, typename Epi>
__device__ __noinline__ void grid_reduce_tail(Reduce red, Epi epi) {
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    acc[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      acc[k] += __ldcg(&red.partials[(size_t)k * red.max_blocks + b]);
  }
  block_sum<NV>(acc);
  if (threadIdx.x == 0) {
    *red.ticket = 0u;
    epi(acc);
  }
}

// Grid-wide deterministic reduction: each block stores its partial sums; the
// last block to finish reduces them (grid_reduce_tail).  Requires
// gridDim.x <= red.max_blocks.
template <int NV, typename Epi>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], Reduce red, Epi epi) {
  __shared__ bool last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red.partials[(size_t)k * red.max_blocks + blockIdx.x] = v[k];
    __threadfence();
    unsigned t = atomicAdd(red.ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) grid_reduce_tail<NV>(red, epi);
}

// ------------------------------------------------------------------ host helpers

int grid_for(int64_t work_items, int threads, int num_sms, int blocks_per_sm);

// Exclusive scans; *total (host) receives the sum when non-null (synchronises).
int scan_exclusive_i32(Arena& ar, const int32_t* in, int32_t* out, int64_t n, int64_t* total,
                       cudaStream_t s);
int scan_exclusive_i64(Arena& ar, const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                       cudaStream_t s);

// SELL conversion (sell.cu)
int sell_from_csr(Arena& ar, int64_t n, int64_t ncols, const int64_t* rowptr, const int32_t* col,
                  const double* val, int C, int tpr, Sell& out, cudaStream_t s,
                  const std::vector<int64_t>* sys_off = nullptr, bool compress = true);
int sell_make_copies(Arena& ar, Sell& A, int vstore, cudaStream_t s);
// Builds A.d16 / A.kbase from A.col (left null when a slice's column offsets
// exceed 16 bits).  Synchronous.
int sell_compress(Arena& ar, Sell& A, cudaStream_t s);
int sell_spmv64(const Sell& A, double alpha, const double* x, double beta, double* y,
                int num_sms, cudaStream_t s);

// Matching and VBM aggregation: the value of edge {i, j} is the entry stored
// in row min(i, j).  Matrices that are symmetric in exact arithmetic need not
// be symmetric bit for bit (smoothed coarse matrices P^T (A P) are not), and
// both endpoints must see the same value.  aij: the entry of row i.  Rows are
// searched by bisection (ascending columns), then by a scan; false when row j
// holds no column i (a structurally unsymmetric pattern: the edge is then not
// eligible).
__device__ __forceinline__ bool edge_value(const int64_t* __restrict__ rowptr,
                                           const int32_t* __restrict__ col,
                                           const double* __restrict__ val, int32_t i, int32_t j,
                                           double aij, double* out) {
  if (j > i) {
    *out = aij;
    return true;
  }
  const int64_t b = rowptr[j], end = rowptr[j + 1];
  int64_t lo = b, hi = end;
  while (lo < hi) {
    const int64_t mid = lo + ((hi - lo) >> 1);
    if (col[mid] < i)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < end && col[lo] == i) {
    *out = val[lo];
    return true;
  }
  for (int64_t e = b; e < end; ++e)
    if (col[e] == i) {
      *out = val[e];
      return true;
    }
  return false;
}

// Matching kernels (setup.cu), also launched by the allocation-free variant
__global__ void k_l1_diag(int64_t n, const int64_t* rowptr, const int32_t* col,
                          const double* val, double* d, double* diag);
// Decoupled Vanek-Mandel-Brezina aggregation (vbm.cu): agg (n, device) gets
// the aggregate of every row, *nc their count, *stride the smallest power of
// two >= the largest aggregate.  diag: a_ii.  AMG_ERR_UNSUPPORTED when rows
// are left for the third phase (structurally unsymmetric patterns).
int vbm_aggregate(Arena& ar, int64_t n, const int64_t* rowptr, const int32_t* col,
                  const double* val, const double* diag, double theta, int32_t* agg, int64_t* nc,
                  int* stride, int num_sms, cudaStream_t s);
__global__ void k_iota(int64_t n, int32_t* a);
__global__ void k_match_cand(const int32_t* __restrict__ wl, const int* __restrict__ nwl,
                             const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ diag,
                             const int32_t* __restrict__ mate, int32_t* __restrict__ cand,
                             int32_t* __restrict__ flag, int* rounds);
__global__ void k_match_commit(const int32_t* __restrict__ wl, const int* __restrict__ nwl,
                               const int32_t* __restrict__ cand, int32_t* mate);
__global__ void k_match_expand(const int32_t* __restrict__ wl, const int* __restrict__ nwl,
                               const int64_t* __restrict__ rowptr,
                               const int32_t* __restrict__ col, const int32_t* __restrict__ mate,
                               int32_t* __restrict__ flag, int32_t* __restrict__ wl_next,
                               int* __restrict__ nwl_next);
__global__ void k_match_final(int64_t n, int32_t* mate);

// Setup (setup.cu)
// like: reuse that hierarchy's aggregates on every level (new values, the
// same structure) instead of matching.
int setup_hierarchy(amg_handle* H, const amg_csr* A, cudaStream_t s,
                    const amg_handle* like = nullptr);
int match_round_loop(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                     const double* diag, int32_t* mate, int32_t* cand, int32_t* flag,
                     int32_t* wl, int64_t wl_stride, int* cnt, int* rounds_out, int num_sms,
                     cudaStream_t s);
// Arguments of a caller's CSR matrix: AMG_ERR_ARG for null pointers or
// sizes that cannot describe one, AMG_ERR_UNSUPPORTED beyond int32 rows.
int check_csr(const amg_csr* A);
int match_pairwise(Arena& ar, int64_t n, const int64_t* rowptr, const int32_t* col,
                   const double* val, int32_t* mate, int* rounds, cudaStream_t s);
int set_level0_weights(amg_handle* H, const float* omega, cudaStream_t s);

// V-cycle (vcycle.cu).  dots: 0 none; 1 (r, z); 2 (r, z) and (z, q).
// r32 (optional, FP32 hierarchies): the same r rounded to float, gathered by
// the level-0 pre-smoother instead of converting every FP64 element.
int vcycle_run(const amg_handle* H, const double* r, double* z, int dots, const double* q,
               cudaStream_t s, double* slice_part = nullptr, const float* r32 = nullptr);
int debug_convert(const double* in64, float* out32, const float* in32, double* out64,
                  int64_t n, cudaStream_t s);
int vcycle_profile(const amg_handle* H, const double* r, double* z, amg_kernel_time* out,
                   int max_out, int* count, cudaStream_t s);
int time_level(const amg_handle* H, int l, int reps, const double* b64, double* z64, float* ms,
               cudaStream_t s);

// Persistent launch of the small levels (tail.cu): levels lt .. coarsest of
// one V-cycle (pre, restrict, coarse solve, post) separated by grid barriers.
// tail_init sizes the grid after setup; tail_start gives lt, or -1 when the
// per-level kernels run every level.  tail_reset clears the barrier after a
// reported timeout.
int tail_init(amg_handle* H, cudaStream_t s);
int tail_start(const amg_handle* H);
template <typename T>
int tail_launch(const amg_handle* H, int lt, cudaStream_t s, const int* act = nullptr);
int tail_reset(amg_handle* H, cudaStream_t s);
// Synchronous: AMG_ERR_DEVICE_CHECK (and a reset) if a persistent launch gave
// up waiting at a barrier, or a streaming kernel gave up waiting for a bulk
// copy, since the last check, else AMG_OK.
int tail_check(amg_handle* H, cudaStream_t s);

// Sparse products for smoothed prolongators (spgemm.cu).  C = X Y with the
// sums of every entry in ascending inner-index order (no fused multiply-
// add); the transpose with ascending columns; P = P_hat - w D^-1 (A P_hat)
// in place over the CSR of A P_hat (columns sorted), w = 1/||D^-1 A||_inf.
int spgemm(Arena& ar, int64_t n, const int64_t* X_rp, const int32_t* X_ci, const double* X_v,
           const int64_t* Y_rp, const int32_t* Y_ci, const double* Y_v, int64_t** C_rp,
           int32_t** C_ci, double** C_v, int64_t* C_nnz, int* dev_status, int num_sms,
           cudaStream_t s);
int transpose_csr(Arena& ar, int64_t n, int64_t ncols, const int64_t* rp, const int32_t* ci,
                  const double* v, int64_t nnz, int64_t** T_rp, int32_t** T_ci, double** T_v,
                  int num_sms, cudaStream_t s);
// A_F of the filtered prolongator smoothing (option prolongator_filter):
// entries with |a_ij| < theta sqrt(a_ii a_jj) dropped, each row's dropped
// entries added to its diagonal; diag = a_ii.
int filter_matrix(Arena& ar, int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                  const double* diag, double theta, int64_t** F_rp, int32_t** F_ci,
                  double** F_v, int num_sms, cudaStream_t s);
int smoothed_prolongator(Arena& ar, int64_t n, const int64_t* A_rp, const int32_t* A_ci,
                         const double* A_v, const int32_t* agg, const int64_t* rp, int32_t* ci,
                         double* v, double* w_out, int num_sms, cudaStream_t s);

// exec = [ctl] -> while (condition) { body; ctl }, where ctl launches the
// kernel that sets the condition through the handle (pcg.cu).
// AMG_ERR_UNSUPPORTED if the runtime cannot build it.
int build_while_graph(cudaStream_t cs, const std::function<int(cudaStream_t)>& body,
                      const std::function<void(cudaStream_t, cudaGraphConditionalHandle)>& ctl,
                      cudaGraphExec_t* out);

// PCG (pcg.cu)
int pcg_run(amg_handle* H, const double* b, double* x, const pcg_options* o, pcg_stats* st,
            cudaStream_t s);

// Multiple right-hand sides (multi.cu)
int vcycle_multi(amg_handle* H, int K, const double* R, double* Z, cudaStream_t s);
int pcg_multi_run(amg_handle* H, int K, const double* B, double* X, const pcg_options* o,
                  pcg_stats* st, cudaStream_t s);
void multi_free(amg_handle* H);

// Two-grid loss for the learned smoother (twogrid.cu)
int twogrid_loss(amg_handle* H, int nsamples, int K, const double* e0, double* loss,
                 float* domega, cudaStream_t s);
void tg_free(amg_handle* H);

// Batched systems (batch.cu)
int concat_systems(Arena& ar, int nsys, const amg_csr* A, amg_csr* cat, int64_t** rp,
                   int32_t** ci, double** va, std::vector<int64_t>& off, int num_sms,
                   cudaStream_t s);
int batch_init(amg_handle* H, cudaStream_t s);
int pcg_batch_run(amg_handle* H, const double* b, double* x, const pcg_options* o, pcg_stats* st,
                  cudaStream_t s);

}  // namespace amg
