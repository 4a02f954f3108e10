// Sliced-ELL row traversal shared by the SpMV, smoother and PCG kernels.
//
// Mapping: one warp per group of R = 32 / TPR consecutive rows (a slice, when
// the slice height C is R).  Lane = t * R + r handles row r of the group and
// the entries k = t, t + TPR, ... of that row, so with C == R every load
// instruction of a warp touches 32 consecutive entries of the column-major
// slice (fully coalesced); with C != R (the autotuner's decoupled layouts) the
// lanes of a row group read C-row runs of one or several slices.  The TPR partial sums of a row are
// combined with xor-shuffles (fixed order).  Matrix values and column indices
// are streamed with evict-first loads; the gathered vectors stay in L2.
#pragma once

#include "common.cuh"

namespace amg {

constexpr int SELL_BLOCK = 256;  // threads per block (8 slices in flight)
// 8 resident blocks per SM (64 warps, full occupancy): at most 32 registers,
// which the streaming kernels need to keep enough loads in flight.
#define SELL_MIN_BLOCKS 8

// Layout code of a SELL kernel instantiation: threads per row (1, 2, 4, 8,
// or 16 and 32 for wide rows) plus SELL_D16 when the matrix stores
// compressed columns (1..8 threads per row only).
constexpr int SELL_D16 = 64;

template <int TPR>
struct Lanes {
  static constexpr int W = TPR & 63;  // threads per row
  static constexpr bool D16 = (TPR & SELL_D16) != 0;
  static constexpr int C = 32 / W;
  int r, t;
  __device__ __forceinline__ Lanes() {
    int lane = threadIdx.x & 31;
    r = lane % C;
    t = lane / C;
  }
};

// sum_k a_{row,k} * g(col_{row,k}) over the entries of this lane's row in
// warp row-group s (32/TPR rows), accumulated in AccT.  When the slice height
// is 32/TPR (one slice per group, every layout but the autotuner's decoupled
// ones, and every batched one) the group is the slice; otherwise each lane
// finds its row's own slice (row i: slice i / C, slot k at
// sliceptr + k C + i mod C), and the row's entries are visited in the same
// order.  Compressed columns (SELL_D16 in the layout code; A.d16 set) give
// the same j for every slot, so the sum is the same bits either way.
//
// NEG: init - sum_k a_k g(col_k) instead, each entry by an FMA with the
// negated value (no separate subtraction); init is added by the row's first
// lane (t == 0) only.
template <int TPR, typename AccT, bool NEG = false, typename V, typename G>
__device__ __forceinline__ AccT sell_row(const SellView<V>& A, int64_t s, const Lanes<TPR>& ln,
                                         G g, AccT init = AccT(0)) {
  constexpr int C = Lanes<TPR>::C, W = Lanes<TPR>::W;
  AccT acc = ln.t == 0 ? init : AccT(0);
  if (!A.row0 && A.C != C) {
    const int64_t i = s * C + ln.r;
    if (i < A.n) {
      const int64_t sl = i / A.C;
      const int64_t b0 = __ldg(A.sliceptr + sl);
      const int w = (int)((__ldg(A.sliceptr + sl + 1) - b0) / A.C);
      const int64_t beg = b0 + (i - sl * A.C);
      const V* vp = A.val + beg;
      if constexpr (Lanes<TPR>::D16) {
        const uint16_t* dp = A.d16 + beg;
        const int32_t* bp = A.kbase + b0 / A.C;
#pragma unroll 4
        for (int k = ln.t; k < w; k += W) {
          const int j = __ldg(bp + k) + (int)ld_stream(dp + (int64_t)k * A.C);
          const AccT a = to_f(ld_stream(vp + (int64_t)k * A.C), AccT(0));
          acc = fma(NEG ? -a : a, g(j), acc);
        }
      } else {
        const int32_t* cp = A.col + beg;
#pragma unroll 4
        for (int k = ln.t; k < w; k += W) {
          const int j = ld_stream(cp + (int64_t)k * A.C);
          const AccT a = to_f(ld_stream(vp + (int64_t)k * A.C), AccT(0));
          acc = fma(NEG ? -a : a, g(j), acc);
        }
      }
    }
#pragma unroll
    for (int o = C; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
  }
  const int64_t beg = __ldg(A.sliceptr + s);
  const int w = (int)((__ldg(A.sliceptr + s + 1) - beg) / C);
  const V* vp = A.val + beg + ln.r;
  if constexpr (Lanes<TPR>::D16) {
    const uint16_t* dp = A.d16 + beg + ln.r;
    const int32_t* bp = A.kbase + beg / C;
#pragma unroll 4
    for (int k = ln.t; k < w; k += W) {
      const int j = __ldg(bp + k) + (int)ld_stream(dp + (int64_t)k * C);
      const AccT a = to_f(ld_stream(vp + (int64_t)k * C), AccT(0));
      acc = fma(NEG ? -a : a, g(j), acc);
    }
  } else {
    const int32_t* cp = A.col + beg + ln.r;
#pragma unroll 4
    for (int k = ln.t; k < w; k += W) {
      const int j = ld_stream(cp + (int64_t)k * C);
      const AccT a = to_f(ld_stream(vp + (int64_t)k * C), AccT(0));
      acc = fma(NEG ? -a : a, g(j), acc);
    }
  }
#pragma unroll
  for (int o = C; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return acc;
}

#define AMG_SELL_CASE(code, ...) \
  case code: {                    \
    constexpr int TPR = code;     \
    __VA_ARGS__;                  \
  } break;

// Runs the statement with TPR = the layout code (see Lanes) as a constant.
#define AMG_DISPATCH_TPR(code, ...)        \
  switch (code) {                          \
    AMG_SELL_CASE(1, __VA_ARGS__)          \
    AMG_SELL_CASE(2, __VA_ARGS__)          \
    AMG_SELL_CASE(4, __VA_ARGS__)          \
    AMG_SELL_CASE(8, __VA_ARGS__)          \
    AMG_SELL_CASE(16, __VA_ARGS__)         \
    AMG_SELL_CASE(32, __VA_ARGS__)         \
    AMG_SELL_CASE(65, __VA_ARGS__)         \
    AMG_SELL_CASE(66, __VA_ARGS__)         \
    AMG_SELL_CASE(68, __VA_ARGS__)         \
    AMG_SELL_CASE(72, __VA_ARGS__)         \
    default:                               \
      return AMG_ERR_ARG;                  \
  }

inline int sell_code(const Sell& A) { return A.tpr | (A.d16 ? SELL_D16 : 0); }

// Warp row-groups of 32/tpr rows that the one-warp-per-group kernels iterate
// over A (see SellView::ngroups).
inline int64_t sell_groups(const Sell& A) {
  const int R = 32 / A.tpr;
  if (A.row0 || A.C == R) return A.nslices;
  return (A.n + R - 1) / R;
}

template <typename V>
inline SellView<V> view(const Sell& A, const V* val) {
  SellView<V> v;
  v.n = A.n;
  v.nslices = A.nslices;
  v.ngroups = sell_groups(A);
  v.C = A.C;
  v.sliceptr = A.sliceptr;
  v.col = A.col;
  v.val = val;
  v.row0 = A.row0;
  v.sys = A.sys;
  v.d16 = A.d16;
  v.kbase = A.kbase;
  v.act = nullptr;
  return v;
}

// Row handled by this lane in warp row-group sl, or -1 (padding lane /
// sub-row lane).
template <int TPR, typename V>
__device__ __forceinline__ int64_t lane_row(const SellView<V>& A, int64_t sl,
                                            const Lanes<TPR>& ln) {
  constexpr int C = Lanes<TPR>::C;
  const int64_t i = A.rbeg(sl, C) + ln.r;
  return (ln.t == 0 && i < A.rend(sl, C)) ? i : -1;
}

// Grid for one-warp-per-group kernels: enough blocks to fill the GPU, capped
// by the group count (grid-stride loop inside).
inline int sell_grid(int64_t ngroups, int num_sms, int blocks_per_sm = 8) {
  return grid_for(ngroups * 32, SELL_BLOCK, num_sms, blocks_per_sm);
}

}  // namespace amg
