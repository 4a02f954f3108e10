// Sliced-ELL streams through a shared-memory ring filled by bulk copies.
//
// The level operators are HBM streams (Sec. 2.1: sparse kernels move O(1)
// bytes per flop), and a warp that loads its slice entry by entry keeps only
// a few loads in flight, so DRAM latency bounds it.  Here every warp owns a
// ring of D stages in shared memory; one lane starts the copy of a whole
// slice (values and column indices, each one contiguous block of the
// column-major slice) with cp.async.bulk, completion counted in bytes on the
// stage's mbarrier, D - 1 slices ahead of the one being consumed.  The lanes
// then read their row's entries from shared memory and gather the vector
// through L2.  Slices of a warp: gw, gw + W, gw + 2W, ... (W warps in the
// grid), the same slice order as the grid-stride kernels.
//
// The slice's 32 entries of the kernel's per-row vectors (b, s, r, the
// aggregate map, ...) come with it, so every DRAM stream of the loop is a
// bulk copy started D - 1 slices ahead; the ragged last slice reads those
// from global memory instead (its copy would run past the vectors' end).
//
// Requirements (checked on the host by ring_plan): one thread per row and
// slice height 32 (lane = row of the slice), one system (no row0), plain
// int32 columns, and a widest slice that fits a stage.  Slice s starts at
// sliceptr[s], a multiple of 32, so both copies start on 16-byte boundaries
// and have sizes that are multiples of 16 bytes (32 w values of 2, 4 or 8
// bytes; 32 w int32 columns); the per-row copies are 32 entries of 4 or 8
// bytes at offset 32 s entries of 256-byte aligned vectors.
//
// Bounded waits: a wait for a stage gives up after RING_WAIT_NS of
// %globaltimer, sets the handle's sticky failure flag, waits (bounded) for
// the warp's other copies in flight and leaves the loop; later launches see
// the flag and return at once, and pcg_solve reports AMG_ERR_DEVICE_CHECK.
#pragma once

#include "sellk.cuh"

namespace amg {

constexpr int RING_WARPS = 8;                      // warps per CTA
constexpr int RING_THREADS = RING_WARPS * 32;
constexpr int RING_MAX_STAGES = 4;
constexpr unsigned long long RING_WAIT_NS = 1000000000ull;  // 1 s
constexpr size_t RING_SMEM_PER_CTA = 112 * 1024;   // at least two CTAs per SM
constexpr int RING_DEFAULT_STAGES = 2;
constexpr size_t RING_ALIGN_SLACK = 128;

constexpr int RING_MAX_ROWS = 5;  // per-row vectors staged with each slice

// Per-row vectors copied into the stage with each slice (the slice's 32
// consecutive entries of each): base pointers and element sizes.
struct RingRows {
  const void* p[RING_MAX_ROWS] = {};
  int esz[RING_MAX_ROWS] = {};
  int n = 0;
  void add(const void* ptr, int bytes) {
    p[n] = ptr;
    esz[n] = bytes;
    ++n;
  }
};

// Ring geometry of one launch (host-computed).  A stage holds the slice's
// values, its columns, then 32 entries of each per-row vector.
struct RingGeom {
  int D = 0;            // stages per warp (0: not eligible)
  uint32_t stage = 0;   // bytes per stage
  uint32_t coff = 0;    // offset of the columns within a stage
  uint32_t roff[RING_MAX_ROWS] = {};  // offsets of the per-row vectors
  int grid = 0;         // CTAs (ring_prepare)
  size_t smem = 0;      // dynamic shared memory per CTA
};

// ------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// The initialised barriers become visible to the async proxy (bulk copies).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_test_parity(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long ring_now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits until the barrier's phase with this parity has completed; false
// after RING_WAIT_NS.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_test_parity(bar, parity)) return true;
  const unsigned long long t0 = ring_now_ns();
  for (;;) {
    if (mbar_test_parity(bar, parity)) return true;
    if (ring_now_ns() - t0 > RING_WAIT_NS) return false;
  }
}

// L2 policy for the matrix streams: evict first, so the gathered vectors
// stay in L2.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completion counted on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                              uint32_t bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1], %2, [%3], %4;" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(pol)
      : "memory");
}

// ------------------------------------------------------------------ per-warp ring

// One warp's ring over the slices gw, gw + nwt, ... of a SELL matrix with
// slice height 32.  Lane 0 issues, every lane consumes.  Usage:
//   RingWarp<V> ring(A, g, smem);  ring.start();
//   for (int64_t sl = ring.first; sl < A.nslices; sl += ring.nwt) {
//     if (!ring.wait()) { ...report...; ring.drain(); break; }  // gave up
//     ... ring.width(), ring.val(k), ring.col(k) of slice sl ...
//     ring.release();                   // stage free: refill with sl + D nwt
//   }
// Every copy issued is consumed before the loop ends, so none is in flight
// when the kernel returns (drain() covers the loop left early).
template <typename V>
struct RingWarp {
  const SellView<V>& A;
  const RingGeom& g;
  const RingRows& rows;
  unsigned char* base;  // this warp's first stage
  uint32_t bar0;        // this warp's first barrier (shared address)
  int* widths;          // per stage: ELL width of the slice it holds
  int64_t first, nwt, cur;
  int stage = 0;
  uint32_t phase = 0;   // parity of the current stage's next completion
  int lane;
  uint64_t pol;
  bool ok = true;
  int64_t nbeg = 0, nend = 0;  // lane 0: bounds of the slice release() copies next

  __device__ __forceinline__ RingWarp(const SellView<V>& A_, const RingGeom& g_,
                                      const RingRows& rows_, unsigned char* smem_raw)
      : A(A_), g(g_), rows(rows_) {
    // 128-byte aligned start (the launch adds RING_ALIGN_SLACK bytes)
    unsigned char* smem =
        smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const int warp = threadIdx.x >> 5;
    lane = threadIdx.x & 31;
    base = smem + (size_t)warp * g.D * g.stage;
    uint64_t* bars = (uint64_t*)(smem + (size_t)RING_WARPS * g.D * g.stage);
    bar0 = smem_addr(bars + warp * RING_MAX_STAGES);
    widths = (int*)(bars + RING_WARPS * RING_MAX_STAGES) + warp * RING_MAX_STAGES;
    nwt = (int64_t)gridDim.x * RING_WARPS;
    first = (int64_t)blockIdx.x * RING_WARPS + warp;
    cur = first;
    pol = l2_evict_first();
  }

  __device__ __forceinline__ uint32_t bar(int d) const { return bar0 + 8u * (uint32_t)d; }

  // Slice sl has 32 rows (not the ragged last slice): its per-row vectors
  // come with it; the last slice's are read from global memory.
  __device__ __forceinline__ bool full(int64_t sl) const { return (sl + 1) * 32 <= A.n; }

  // lane 0: copy slice sl = [beg, end) (and its per-row vectors) into stage d
  __device__ __forceinline__ void issue(int64_t sl, int d, int64_t beg, int64_t end) {
    const int w = (int)((end - beg) >> 5);
    widths[d] = w;
    const uint32_t vb = (uint32_t)w * 32u * (uint32_t)sizeof(V), cb = (uint32_t)w * 128u;
    const bool f = full(sl);
    uint32_t rb = 0;
#pragma unroll
    for (int k = 0; k < RING_MAX_ROWS; ++k)
      if (f && k < rows.n) rb += 32u * (uint32_t)rows.esz[k];
    const uint32_t dst = smem_addr(base + (size_t)d * g.stage);
    mbar_arrive_expect_tx(bar(d), vb + cb + rb);
    if (w > 0) {
      bulk_copy_g2s(dst, A.val + beg, vb, bar(d), pol);
      bulk_copy_g2s(dst + g.coff, A.col + beg, cb, bar(d), pol);
    }
#pragma unroll
    for (int k = 0; k < RING_MAX_ROWS; ++k)
      if (f && k < rows.n)
        bulk_copy_g2s(dst + g.roff[k], (const unsigned char*)rows.p[k] + sl * 32 * rows.esz[k],
                      32u * (uint32_t)rows.esz[k], bar(d), pol);
  }

  // barriers initialised, the first D slices on their way
  __device__ __forceinline__ void start() {
    if (lane == 0) {
      for (int d = 0; d < g.D; ++d) mbar_init(bar(d), 1);
      mbar_init_fence();
      for (int d = 0; d < g.D; ++d) {
        const int64_t sl = first + (int64_t)d * nwt;
        if (sl < A.nslices) issue(sl, d, __ldg(A.sliceptr + sl), __ldg(A.sliceptr + sl + 1));
      }
    }
    __syncwarp();
  }

  // Waits for the current slice.  Lane 0 first loads the bounds of the slice
  // that release() will copy next, so that load's latency passes during the
  // wait and the slice's arithmetic instead of delaying the copy.
  __device__ __forceinline__ bool wait() {
    const int64_t nxt = cur + (int64_t)g.D * nwt;
    if (lane == 0 && nxt < A.nslices) {
      nbeg = __ldg(A.sliceptr + nxt);
      nend = __ldg(A.sliceptr + nxt + 1);
    }
    ok = mbar_wait_bounded(bar(stage), phase);
    return __all_sync(0xffffffffu, ok);
  }

  __device__ __forceinline__ int width() const { return widths[stage]; }
  __device__ __forceinline__ V val(int k) const {
    return ((const V*)(base + (size_t)stage * g.stage))[k * 32 + lane];
  }
  __device__ __forceinline__ int32_t col(int k) const {
    return ((const int32_t*)(base + (size_t)stage * g.stage + g.coff))[k * 32 + lane];
  }
  // entry i = 32 cur + lane of per-row vector k (element type X = its type)
  template <typename X>
  __device__ __forceinline__ X row(int k, bool f, int64_t i) const {
    if (f) return ((const X*)(base + (size_t)stage * g.stage + g.roff[k]))[lane];
    return __ldg((const X*)rows.p[k] + i);
  }

  // every lane is done with the current stage: refill it, move on
  __device__ __forceinline__ void release() {
    __syncwarp();
    const int64_t nxt = cur + (int64_t)g.D * nwt;
    if (lane == 0 && nxt < A.nslices) issue(nxt, stage, nbeg, nend);
    cur += nwt;
    if (++stage == g.D) {
      stage = 0;
      phase ^= 1u;
    }
  }

  // After a wait that gave up: wait (bounded) for the copies still in
  // flight, so none lands in shared memory after the CTA has exited.
  __device__ __forceinline__ void drain() {
    for (int d = 0; d < g.D; ++d) {
      const int64_t sl = cur + (int64_t)d * nwt;
      if (sl >= A.nslices) break;
      const int st = (stage + d) % g.D;
      const uint32_t ph = phase ^ (uint32_t)((stage + d) / g.D);
      if (!mbar_wait_bounded(bar(st), ph)) break;
    }
  }
};

// acc + sum of a_k g(col_k) (NEG: acc - sum, by FMAs with the negated
// values) for k = k0 .. k0 + N - 1, k ascending: the N gathers issue
// together, then the FMAs follow in order.  Exactly N FMAs: on GB300's FP64
// pipe a predicated-off FMA would still cost its cycles.
template <int N, bool NEG, typename T, typename V, typename G>
__device__ __forceinline__ T ring_chunk(const RingWarp<V>& ring, int k0, T acc, G g) {
  T x[N];
#pragma unroll
  for (int u = 0; u < N; ++u) x[u] = g(ring.col(k0 + u));
#pragma unroll
  for (int u = 0; u < N; ++u) {
    const T a = to_f(ring.val(k0 + u), T(0));
    acc = fma(NEG ? -a : a, x[u], acc);
  }
  return acc;
}

// init + sum_k a_k g(col_k) (NEG: init - sum) over the w entries of this
// lane's row in the current stage, k ascending (the per-lane kernels'
// order): chunks of 8 and one remainder chunk of the exact length (w is
// warp-uniform).
template <typename T, bool NEG = false, typename V, typename G>
__device__ __forceinline__ T ring_row_sum(const RingWarp<V>& ring, int w, G g, T init = T(0)) {
  T acc = init;
  int k0 = 0;
  for (; k0 + 8 <= w; k0 += 8) acc = ring_chunk<8, NEG>(ring, k0, acc, g);
  switch (w - k0) {
    case 1: acc = ring_chunk<1, NEG>(ring, k0, acc, g); break;
    case 2: acc = ring_chunk<2, NEG>(ring, k0, acc, g); break;
    case 3: acc = ring_chunk<3, NEG>(ring, k0, acc, g); break;
    case 4: acc = ring_chunk<4, NEG>(ring, k0, acc, g); break;
    case 5: acc = ring_chunk<5, NEG>(ring, k0, acc, g); break;
    case 6: acc = ring_chunk<6, NEG>(ring, k0, acc, g); break;
    case 7: acc = ring_chunk<7, NEG>(ring, k0, acc, g); break;
    default: break;
  }
  return acc;
}

// A bounded wait gave up: the handle's sticky flag, and the PCG status
// (if given) so a device-side loop stops.
__device__ __forceinline__ void ring_fail(int* fail, int* status) {
  atomicExch(fail, 1);
  if (status) atomicCAS(status, 0, AMG_ERR_DEVICE_CHECK);
}

// Geometry for streaming M (values of `vbytes` bytes) with the ring, or
// D = 0 when M does not qualify.  stages: 2..RING_MAX_STAGES, or 0 for the
// default.  The grid is left to ring_launch_grid.  Host code.
RingGeom ring_plan(const Sell& M, int vbytes, int stages, const RingRows& rows);

// Prepares kernel `fn` for a launch with geometry g on the current device
// (shared-memory limit, once per device and kernel) and sets g.grid to the
// CTAs that are co-resident (occupancy query), at most one slice per warp.
// Host code.
int ring_prepare(const void* fn, RingGeom& g, int64_t nslices, int num_sms);

}  // namespace amg
