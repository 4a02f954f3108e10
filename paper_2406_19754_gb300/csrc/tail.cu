// The small levels of the V(1,1) cycle in one persistent launch.
//
// Below a few hundred thousand rows a level's pre-smoother, restriction and
// post-smoother each move only a few MB, so one kernel per step costs mostly
// launch latency.  Here levels lt .. coarsest run in one cooperative launch:
//
//   for l = lt .. L-2:  r_l = b_l - Ah_l b_l  | barrier |  b_{l+1} = P^T r_l  | barrier |
//   coarsest:           x = L^-T (L^-1 b)     | barrier |
//   for l = L-2 .. lt:  x_l = S b_l + P x_{l+1} + S (r_l - AP_l x_{l+1})  | barrier |
//
// with the same per-row code as the one-kernel-per-step path (smooth.cuh),
// so results are identical bit for bit.  Vectors written inside the launch
// are read through L2 (ld.global.cg), never through the read-only cache.
//
// The grid barrier: every CTA adds to one counter, CTA 0 adds 2^31 - (G-1)
// and the others 1, so the counter's top bit flips once all G have arrived;
// each CTA waits for the flip.  The cooperative launch guarantees that all
// CTAs are resident.  A wait longer than one second (which a correct launch
// never reaches) sets a sticky failure flag, reports AMG_ERR_DEVICE_CHECK in
// the PCG status and the handle's device status, and the CTA returns; later
// launches return at once until tail_reset clears the flag and the counter.
// A test hook (amg_debug_tail_timeout) makes CTA 0 count one arrival that
// never comes, so every wait runs out after 10 ms and that path is exercised.
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "smooth.cuh"

namespace amg {

namespace {

constexpr int TAIL_BLOCK = 1024;
constexpr int TAIL_MAX_LEVELS = 16;
constexpr int TAIL_MAX_PREFETCH = 64;
// A tail whose largest level has at most this many rows runs in one CTA.
constexpr int64_t TAIL_ONE_CTA_ROWS = 16384;
constexpr unsigned long long TAIL_WAIT_NS = 1000000000ull;        // 1 s
constexpr unsigned long long TAIL_DEBUG_WAIT_NS = 10000000ull;    // 10 ms (test hook)

struct SellDesc {
  int64_t n, nslices, ngroups;
  int C;
  const int64_t* sliceptr;
  const int32_t* col;
  const void* val;
  const int64_t* row0;
  const int32_t* sys;
  const uint16_t* d16;
  const int32_t* kbase;
  const int* act;
  int tpr;
};

struct TailLevel {
  SellDesc A, AP;  // Ah = A S and AP = A P in the level's value storage
  int vstore, stride;
  int64_t nc;
  const void* s;
  const int32_t* agg;
  const int32_t* members;
  void *b, *x, *r;  // this level
  void* bc;         // next level's b
  const void* xc;   // next level's x
  int64_t nu;       // smoother sweeps; with nu > 1 also r2 and the pre-smoothed xp
  void *r2, *xp;
};

struct TailParams {
  int nlev;   // smoothed levels lt .. lt + nlev - 1; the next one is the coarsest
  int small;  // coarsest blocks solved one per CTA (else row-parallel, two phases)
  // coarsest solve by PCG-l1 (one CTA only): its matrix, scale and scratch
  int pcg, pcg_maxit;
  double pcg_tol;
  SellDesc Ac;
  const double* csinv;
  double* cw;
  int nblk;
  int64_t nco;
  const int64_t* brow;
  const int64_t* bmat;
  const double* Linv;
  const double* LinvT;
  double* y;
  const void* cb;
  void* cx;
  const int* act;  // batched PCG: per-system active flags (coarse block = system), or null
  unsigned* bar;
  unsigned unreachable;  // test hook: arrivals the barrier waits for that never come
  unsigned long long wait_ns;
  int* fail;
  int* status;      // PCG status word
  int* dev_status;  // handle status word
  // arrays the launch reads, prefetched into L2 at its start (16-byte
  // aligned starts, sizes rounded down to 16 bytes)
  int npf;
  const void* pf_ptr[TAIL_MAX_PREFETCH];
  unsigned pf_bytes[TAIL_MAX_PREFETCH];
  TailLevel lv[TAIL_MAX_LEVELS];
};

template <typename V>
__device__ __forceinline__ SellView<V> dview(const SellDesc& d) {
  SellView<V> v;
  v.n = d.n;
  v.nslices = d.nslices;
  v.ngroups = d.ngroups;
  v.C = d.C;
  v.sliceptr = d.sliceptr;
  v.col = d.col;
  v.val = (const V*)d.val;
  v.row0 = d.row0;
  v.sys = d.sys;
  v.d16 = d.d16;
  v.kbase = d.kbase;
  v.act = d.act;
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier; false if this CTA gave up waiting or a failure is flagged.
__device__ __noinline__ bool tail_sync(const TailParams& P) {
  unsigned* bar = P.bar;
  int* fail = P.fail;
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned inc =
        blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) - P.unreachable : 1u;
    __threadfence();
    const unsigned old = atomicAdd(bar, inc);
    int ok = 1;
    const unsigned long long t0 = global_ns();
    while (((*(volatile unsigned*)bar ^ old) & 0x80000000u) == 0u) {
      if (global_ns() - t0 > P.wait_ns) {
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    if (!ok)
      atomicExch(fail, 1);
    else if (*(volatile int*)fail)
      ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ void tail_report(const TailParams& P) {
  if (P.status) atomicCAS(P.status, 0, AMG_ERR_DEVICE_CHECK);
  atomicExch(P.dev_status, AMG_ERR_DEVICE_CHECK);
}

// ------------------------------------------------------------------ phases

// Layout code of a level's matrix (threads per row, plus SELL_D16 for
// compressed columns); the host builds no other codes.
#define TAIL_TPR(code, ...)         \
  switch (code) {                   \
    AMG_SELL_CASE(1, __VA_ARGS__)   \
    AMG_SELL_CASE(2, __VA_ARGS__)   \
    AMG_SELL_CASE(4, __VA_ARGS__)   \
    AMG_SELL_CASE(8, __VA_ARGS__)   \
    AMG_SELL_CASE(16, __VA_ARGS__)  \
    AMG_SELL_CASE(32, __VA_ARGS__)  \
    AMG_SELL_CASE(65, __VA_ARGS__)  \
    AMG_SELL_CASE(66, __VA_ARGS__)  \
    AMG_SELL_CASE(68, __VA_ARGS__)  \
    AMG_SELL_CASE(72, __VA_ARGS__)  \
    default:                        \
      break;                        \
  }

__device__ __forceinline__ int dcode(const SellDesc& d) {
  return d.tpr | (d.d16 ? SELL_D16 : 0);
}

template <int TPR, typename Ld, typename T, typename V>
__device__ __forceinline__ void pre_rows(const TailLevel& L, int64_t gw, int64_t nw) {
  const Lanes<TPR> ln;
  const SellView<V> Ah = dview<V>(L.A);
  for (int64_t sl = gw; sl < Ah.ngroups; sl += nw)
    if (Ah.live(sl)) pre_slice<TPR, Ld>(Ah, (const T*)L.b, (T*)L.r, sl, ln);
}

template <int TPR, typename Ld, typename T, typename V>
__device__ __forceinline__ void post_rows(const TailLevel& L, const T* r, const T* xp, T* e,
                                          int64_t gw, int64_t nw) {
  const Lanes<TPR> ln;
  const SellView<V> AP = dview<V>(L.AP);
  for (int64_t sl = gw; sl < AP.ngroups; sl += nw) {
    if (!AP.live(sl)) continue;
    T z;
    post_slice<TPR, Ld>(AP, (const T*)L.b, (const T*)L.s, r, L.agg, (const T*)L.xc, (T*)L.x,
                        sl, ln, z, xp, e);
  }
}

// Further sweeps on the residual recurrence (k_sweep_pre / k_sweep_post).
template <int TPR, typename Ld, typename T, typename V, bool PRE>
__device__ __forceinline__ void sweep_rows(const TailLevel& L, const T* r, T* r_out, int first,
                                           int64_t gw, int64_t nw) {
  const Lanes<TPR> ln;
  const SellView<V> Ah = dview<V>(L.A);
  const T* s = (const T*)L.s;
  for (int64_t sl = gw; sl < Ah.ngroups; sl += nw) {
    if (!Ah.live(sl)) continue;
    T ri = T(0), rn = T(0);
    int64_t i;
    sweep_slice<TPR, Ld>(Ah, s, r, r_out, sl, ln, ri, rn, i);
    if (i < 0) continue;
    if constexpr (PRE) {
      T* x = (T*)L.xp;
      const T xi = first ? s[i] * Ld::ld((const T*)L.b + i) : x[i];
      x[i] = sweep_pre_x(xi, s[i], ri);
    } else {
      T* y = (T*)L.x;
      y[i] = sweep_post_y(y[i], s[i], rn);
    }
  }
}

template <typename Ld, typename T>
__device__ void tail_pre(const TailLevel& L, int64_t gw, int64_t nw) {
  if constexpr (sizeof(T) == 8) {
    TAIL_TPR(dcode(L.A), (pre_rows<TPR, Ld, T, double>(L, gw, nw)));
  } else if (L.vstore == VAL_BF16) {
    TAIL_TPR(dcode(L.A), (pre_rows<TPR, Ld, T, __nv_bfloat16>(L, gw, nw)));
  } else {
    TAIL_TPR(dcode(L.A), (pre_rows<TPR, Ld, T, float>(L, gw, nw)));
  }
}

template <typename Ld, typename T>
__device__ void tail_post(const TailLevel& L, const T* r, const T* xp, T* e, int64_t gw,
                          int64_t nw) {
  if constexpr (sizeof(T) == 8) {
    TAIL_TPR(dcode(L.AP), (post_rows<TPR, Ld, T, double>(L, r, xp, e, gw, nw)));
  } else if (L.vstore == VAL_BF16) {
    TAIL_TPR(dcode(L.AP), (post_rows<TPR, Ld, T, __nv_bfloat16>(L, r, xp, e, gw, nw)));
  } else {
    TAIL_TPR(dcode(L.AP), (post_rows<TPR, Ld, T, float>(L, r, xp, e, gw, nw)));
  }
}

template <typename Ld, typename T, bool PRE>
__device__ void tail_sweep(const TailLevel& L, const T* r, T* r_out, int first, int64_t gw,
                           int64_t nw) {
  if constexpr (sizeof(T) == 8) {
    TAIL_TPR(dcode(L.A), (sweep_rows<TPR, Ld, T, double, PRE>(L, r, r_out, first, gw, nw)));
  } else if (L.vstore == VAL_BF16) {
    TAIL_TPR(dcode(L.A),
             (sweep_rows<TPR, Ld, T, __nv_bfloat16, PRE>(L, r, r_out, first, gw, nw)));
  } else {
    TAIL_TPR(dcode(L.A), (sweep_rows<TPR, Ld, T, float, PRE>(L, r, r_out, first, gw, nw)));
  }
}

template <typename Ld, typename T>
__device__ void tail_restrict(const TailLevel& L, const T* r, int64_t gt, int64_t nt) {
  T* bc = (T*)L.bc;
  for (int64_t I = gt; I < L.nc; I += nt)
    bc[I] = restrict_sum<Ld>(L.members + I * L.stride, L.stride, r);
}

// One CTA (ONE): the barrier is __syncthreads and vectors are read with plain
// loads; the grid: the bounded grid barrier and L2-coherent loads.
template <bool ONE>
__device__ __forceinline__ bool tail_barrier(const TailParams& P) {
  if constexpr (ONE) {
    __syncthreads();
    return true;
  } else {
    return tail_sync(P);
  }
}

// Returns false on a barrier failure (reported by the caller).
template <bool ONE, typename Ld, typename T>
__device__ bool tail_coarse(const TailParams& P, int64_t gw, int64_t nw, double* csh) {
  const T* b = (const T*)P.cb;
  T* x = (T*)P.cx;
  if constexpr (ONE) {
    if (P.pcg) {
      const SellView<double> Ac = dview<double>(P.Ac);
      TAIL_TPR(dcode(P.Ac), (coarse_pcg_cta<TPR>(Ac, P.csinv, b, x, P.cw, P.pcg_maxit,
                                                  P.pcg_tol)));
      return true;
    }
  }
  if (P.small) {
    for (int blk = blockIdx.x; blk < P.nblk; blk += gridDim.x)
      if (!P.act || P.act[blk])
        coarse_block_solve<Ld>(blk, P.brow, P.bmat, P.Linv, P.LinvT, b, x, csh);
    return true;
  }
  for (int64_t g = gw; g < P.nco; g += nw)
    coarse_y_row<Ld>(g, P.nblk, P.brow, P.bmat, P.Linv, b, P.y);
  if (!tail_barrier<ONE>(P)) return false;
  for (int64_t g = gw; g < P.nco; g += nw)
    coarse_x_row<Ld>(g, P.nblk, P.brow, P.bmat, P.LinvT, P.y, x);
  return true;
}

template <typename T, bool ONE>
__global__ void __launch_bounds__(TAIL_BLOCK, 1) k_tail(const __grid_constant__ TailParams P) {
  using Ld = typename std::conditional<ONE, LdPlain, LdL2>::type;
  extern __shared__ double csh[];
  if (!ONE && *(volatile int*)P.fail) {
    if (threadIdx.x == 0) tail_report(P);
    return;
  }
  // The small levels' arrays have usually left L2 since the last V-cycle
  // (the level-0 streams pass through it): request all of them at once, so
  // the dependent loads of each phase wait for L2 instead of DRAM.
  if (blockIdx.x == 0 && threadIdx.x < P.npf)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(P.pf_ptr[threadIdx.x]),
                 "r"(P.pf_bytes[threadIdx.x])
                 : "memory");
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  const int64_t gw = gt >> 5, nw = nt >> 5;
  // bit l of cur: which residual buffer of level l (r or r2) holds its
  // residual after the pre-smoothing sweeps
  unsigned cur = 0;
  auto rb = [&](const TailLevel& L, int k) { return (T*)(k ? L.r2 : L.r); };
  bool ok = true;
  for (int l = 0; ok && l < P.nlev; ++l) {
    const TailLevel& L = P.lv[l];
    tail_pre<Ld, T>(L, gw, nw);
    ok = tail_barrier<ONE>(P);
    int c = 0;
    for (int64_t k = 2; ok && k <= L.nu; ++k) {
      tail_sweep<Ld, T, true>(L, rb(L, c), rb(L, 1 - c), k == 2, gw, nw);
      ok = tail_barrier<ONE>(P);
      c = 1 - c;
    }
    if (!ok) break;
    if (c) cur |= 1u << l;
    tail_restrict<Ld, T>(L, rb(L, c), gt, nt);
    ok = tail_barrier<ONE>(P);
  }
  if (ok) ok = tail_coarse<ONE, Ld, T>(P, gw, nw, csh);
  if (ok) ok = tail_barrier<ONE>(P);
  for (int l = P.nlev - 1; ok && l >= 0; --l) {
    const TailLevel& L = P.lv[l];
    int c = (cur >> l) & 1u;
    if (L.nu > 1) {
      tail_post<Ld, T>(L, rb(L, c), (const T*)L.xp, rb(L, 1 - c), gw, nw);
      c = 1 - c;
    } else {
      tail_post<Ld, T>(L, (const T*)L.r, nullptr, nullptr, gw, nw);
    }
    for (int64_t m = 2; ok && m <= L.nu; ++m) {
      ok = tail_barrier<ONE>(P);
      if (!ok) break;
      tail_sweep<Ld, T, false>(L, rb(L, c), rb(L, 1 - c), 0, gw, nw);
      c = 1 - c;
    }
    if (ok && l > 0) ok = tail_barrier<ONE>(P);
  }
  if (!ok && threadIdx.x == 0) tail_report(P);
}

}  // namespace

// ------------------------------------------------------------------ host

static SellDesc desc(const Sell& A, const void* val, const int* act) {
  SellDesc d;
  d.n = A.n;
  d.nslices = A.nslices;
  d.ngroups = sell_groups(A);
  d.C = A.C;
  d.sliceptr = A.sliceptr;
  d.col = A.col;
  d.val = val;
  d.row0 = A.row0;
  d.sys = A.sys;
  d.d16 = A.d16;
  d.kbase = A.kbase;
  d.act = act;
  d.tpr = A.tpr;
  return d;
}

static int64_t largest_coarse_block(const amg_handle* H) {
  int64_t m = 0;
  for (int k = 0; k < H->nblk; ++k) m = std::max(m, H->cblk_row[k + 1] - H->cblk_row[k]);
  return m;
}

int tail_init(amg_handle* H, cudaStream_t s) {
  H->tail_grid = 0;
  if (!H->tail_bar) {
    AMG_TRY(H->arena.alloc_n(&H->tail_bar, 1));
    AMG_TRY(H->arena.alloc_n(&H->tail_fail, 1));
    AMG_CUDA_TRY(cudaMemsetAsync(H->tail_bar, 0, sizeof(unsigned), s));
    AMG_CUDA_TRY(cudaMemsetAsync(H->tail_fail, 0, sizeof(int), s));
  }
  int coop = 0;
  AMG_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, H->device));
  if (!coop) return AMG_OK;
  const size_t smem = sizeof(double) * 2 * (size_t)COARSE_SMALL;
  int occ = 0;
  if (H->opt.precision == AMG_PREC_F32)
    AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tail<float, false>,
                                                               TAIL_BLOCK, smem));
  else
    AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tail<double, false>,
                                                               TAIL_BLOCK, smem));
  H->tail_grid = std::min(occ, 1) * H->num_sms;
  return AMG_OK;
}

int tail_start(const amg_handle* H) {
  const int nl = (int)H->L.size();
  if (H->opt.tail_rows <= 0 || H->tail_grid <= 0 || nl < 3) return -1;
  if (H->opt.smooth_prolongator) return -1;  // the tail restricts and prolongs by aggregates
  int lt = 1;
  while (lt < nl - 1 && H->L[lt].n > H->opt.tail_rows) ++lt;
  lt = std::max(lt, nl - 1 - TAIL_MAX_LEVELS);
  if (lt > nl - 2) return -1;
  // the PCG coarsest solve runs inside a one-CTA tail only
  if (H->opt.coarse_solver != 0 && (H->L[lt].n > TAIL_ONE_CTA_ROWS || H->nblk != 1)) return -1;
  return lt;
}

int tail_reset(amg_handle* H, cudaStream_t s) {
  if (!H->tail_bar) return AMG_OK;
  AMG_CUDA_TRY(cudaMemsetAsync(H->tail_bar, 0, sizeof(unsigned), s));
  AMG_CUDA_TRY(cudaMemsetAsync(H->tail_fail, 0, sizeof(int), s));
  return AMG_OK;
}

int tail_check(amg_handle* H, cudaStream_t s) {
  int f[2] = {0, 0};
  if (H->tail_fail)
    AMG_CUDA_TRY(cudaMemcpyAsync(&f[0], H->tail_fail, sizeof(int), cudaMemcpyDeviceToHost, s));
  // the streaming kernels' flag (ring.cuh): a bounded wait for a bulk copy gave up
  if (H->wait_fail)
    AMG_CUDA_TRY(cudaMemcpyAsync(&f[1], H->wait_fail, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  if (!f[0] && !f[1]) return AMG_OK;
  if (f[0]) AMG_TRY(tail_reset(H, s));
  if (f[1]) {
    // launches that returned early skipped their grid reductions
    AMG_CUDA_TRY(cudaMemsetAsync(H->wait_fail, 0, sizeof(int), s));
    AMG_CUDA_TRY(cudaMemsetAsync(H->red.ticket, 0, sizeof(unsigned), s));
  }
  return AMG_ERR_DEVICE_CHECK;
}

template <typename T>
int tail_launch(const amg_handle* H, int lt, cudaStream_t s, const int* act) {
  const int nl = (int)H->L.size();
  if (lt < 1 || lt > nl - 2 || nl - 1 - lt > TAIL_MAX_LEVELS || H->tail_grid <= 0)
    return AMG_ERR_ARG;
  const bool f64 = sizeof(T) == 8;
  TailParams P;
  memset(&P, 0, sizeof(P));
  P.nlev = nl - 1 - lt;
  int64_t warps = 0;  // most warps any phase can use
  for (int k = 0; k < P.nlev; ++k) {
    const Level& L = H->L[lt + k];
    TailLevel& d = P.lv[k];
    const void* ah = f64 ? (const void*)L.ah64
                         : L.vstore == VAL_BF16 ? (const void*)L.ah16 : (const void*)L.ah32;
    const void* ap = f64 ? (const void*)L.AP.v64
                         : L.vstore == VAL_BF16 ? (const void*)L.AP.v16 : (const void*)L.AP.v32;
    d.A = desc(L.A, ah, act);
    d.AP = desc(L.AP, ap, act);
    d.vstore = L.vstore;
    d.stride = L.stride;
    d.nc = L.nc;
    d.s = f64 ? (const void*)L.s64 : (const void*)L.s32;
    d.agg = L.agg;
    d.members = L.members;
    d.b = L.b;
    d.x = L.x;
    d.r = L.r;
    d.bc = H->L[lt + k + 1].b;
    d.xc = H->L[lt + k + 1].x;
    d.nu = L.nu;
    d.r2 = L.r2;
    d.xp = L.xp;
    warps = std::max({warps, sell_groups(L.A), sell_groups(L.AP), (L.nc + 31) / 32});
  }
  const Level& Lc = H->L[nl - 1];
  const int64_t m = largest_coarse_block(H);
  P.small = m <= COARSE_SMALL ? 1 : 0;
  P.nblk = H->nblk;
  P.nco = H->nco;
  P.brow = H->d_brow;
  P.bmat = H->d_bmat;
  P.Linv = H->Linv;
  P.LinvT = H->LinvT;
  P.y = H->coarse_y;
  P.cb = Lc.b;
  P.cx = Lc.x;
  P.act = act;
  if (H->opt.coarse_solver != 0) {
    P.pcg = 1;
    P.pcg_maxit = H->opt.coarse_maxit;
    P.pcg_tol = H->opt.coarse_tol;
    P.Ac = desc(Lc.A, Lc.A.v64, nullptr);
    P.csinv = Lc.s64;
    P.cw = H->cpcg;
  }
  P.bar = H->tail_bar;
  P.unreachable = H->tail_debug ? 1u : 0u;
  P.wait_ns = H->tail_debug ? TAIL_DEBUG_WAIT_NS : TAIL_WAIT_NS;
  P.fail = H->tail_fail;
  P.status = &H->sc->status;
  P.dev_status = H->dev_status;
  warps = std::max(warps, P.small ? (int64_t)P.nblk * (TAIL_BLOCK / 32) : P.nco);
  auto pf = [&](const void* p, double bytes) {
    const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const double b = bytes - (double)(a - (uintptr_t)p);
    if (!p || b < 16.0 || P.npf >= TAIL_MAX_PREFETCH) return;
    const double cap = 4294967280.0;  // largest multiple of 16 below 2^32
    P.pf_ptr[P.npf] = (const void*)a;
    P.pf_bytes[P.npf] = (unsigned)((uint64_t)std::min(b, cap) & ~(uint64_t)15);
    ++P.npf;
  };
  const double vb = sizeof(T);
  for (int k = 0; k < P.nlev; ++k) {
    const Level& L = H->L[lt + k];
    const double mb = L.vstore == VAL_F64 ? 8.0 : L.vstore == VAL_F32 ? 4.0 : 2.0;
    for (const Sell* M : {&L.A, &L.AP}) {
      pf(M->sliceptr, 8.0 * (double)(M->nslices + 1));
      if (M->d16) {
        pf(M->d16, 2.0 * (double)M->nnz_pad);
        pf(M->kbase, 4.0 * (double)(M->nnz_pad / M->C));
      } else {
        pf(M->col, 4.0 * (double)M->nnz_pad);
      }
    }
    pf(P.lv[k].A.val, mb * (double)L.A.nnz_pad);
    pf(P.lv[k].AP.val, mb * (double)L.AP.nnz_pad);
    pf(P.lv[k].s, vb * (double)L.n);
    pf(L.agg, 4.0 * (double)L.n);
    pf(L.members, 4.0 * (double)L.nc * (double)L.stride);
  }
  {
    double fac = 0.0;  // every diagonal block's L^-1 (and L^-T): contiguous
    for (int k = 0; k < H->nblk; ++k) {
      const double mm = (double)(H->cblk_row[k + 1] - H->cblk_row[k]);
      fac += mm * mm * 8.0;
    }
    pf(H->Linv, fac);
    pf(H->LinvT, fac);
  }
  // small enough for one CTA: no grid barrier at all
  const bool one = H->L[lt].n <= TAIL_ONE_CTA_ROWS && P.nblk == 1;
  if (P.pcg && !one) return AMG_ERR_ARG;
  const int64_t want = (warps * 32 + TAIL_BLOCK - 1) / TAIL_BLOCK;
  const int grid = one ? 1 : (int)std::max<int64_t>(1, std::min<int64_t>(want, H->tail_grid));
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(TAIL_BLOCK);
  cfg.dynamicSmemBytes = P.small ? sizeof(double) * 2 * (size_t)m : 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = one ? 0 : 1;
  if (one)
    AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tail<T, true>, P));
  else
    AMG_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tail<T, false>, P));
  return AMG_OK;
}

template int tail_launch<float>(const amg_handle*, int, cudaStream_t, const int*);
template int tail_launch<double>(const amg_handle*, int, cudaStream_t, const int*);

}  // namespace amg

extern "C" int amg_debug_tail_timeout(amg_handle* H, int on) {
  if (!H) return AMG_ERR_ARG;
  H->tail_debug = on ? 1 : 0;
  // captured iterations hold the launch parameters: capture again
  if (H->graph) cudaGraphExecDestroy(H->graph);
  if (H->bgraph) cudaGraphExecDestroy(H->bgraph);
  if (H->loop) cudaGraphExecDestroy(H->loop);
  if (H->bloop) cudaGraphExecDestroy(H->bloop);
  H->graph = nullptr;
  H->bgraph = nullptr;
  H->loop = nullptr;
  H->bloop = nullptr;
  return AMG_OK;
}
