// Multi-RHS PCG: K independent CG iterations on the same matrix, vectors
// stored row-major N x K so one row's K values are contiguous.
//
// Mapping: one warp per matrix row, lane l owning right-hand sides l and
// l + 32 (KPL = 1 or 2 columns per lane, K <= 64).  Every matrix entry is
// loaded once per warp and applied to all K columns, so the matrix stream is
// amortised K-fold and the kernels stream the N x K vectors.  Per column the
// arithmetic follows the single-RHS kernels' operation order (entries in
// slice order, one FMA each), so the blocked V-cycle reproduces K separate
// V-cycles bit for bit.  Column dot products are reduced per block and then
// by the last block, in fixed order.  Each column has its own alpha, beta and
// stopping test; converged columns are frozen (alpha = 0, p unchanged).
#include <math.h>

#include <algorithm>

#include "sellk.cuh"

namespace amg {

constexpr int MROWS_BLOCK = 256;  // 8 warps = 8 rows in flight per block

struct MultiWs {
  int K = 0;
  double *R = nullptr, *Z = nullptr, *P = nullptr, *Q = nullptr;  // N x K
  float* R32 = nullptr;  // FP32 copy of R for an FP32 V-cycle (else null)
  void** lb = nullptr;  // per level b, x, r (V-cycle type), host arrays of pointers
  void** lx = nullptr;
  void** lr = nullptr;
  double* cy = nullptr;  // coarse scratch n_c x K
  double* part = nullptr;  // 2 x max_blocks x K
  unsigned* ticket = nullptr;
  Scal* sc = nullptr;  // K
  Scal* sc_host = nullptr;
  int* nactive = nullptr;
};

// Entries of row i of a (non-batched) sliced-ELL matrix.
struct RowSpan {
  const int32_t* col;
  int64_t stride;
  int w;
  int64_t off;
};

template <typename V>
__device__ __forceinline__ RowSpan row_span(const SellView<V>& A, int64_t i, int C) {
  const int64_t s = i / C;
  const int64_t beg = __ldg(A.sliceptr + s);
  RowSpan r;
  r.w = (int)((__ldg(A.sliceptr + s + 1) - beg) / C);
  r.off = beg + (i - s * C);
  r.stride = C;
  r.col = A.col;
  return r;
}

// acc[c] = sum_k a_ik * g(col_k, c) for the lane's columns.  Entries go in
// groups of MV_U: the group's columns and values are loaded first, then all
// its gathers are issued, then the FMAs run in entry order, so a warp keeps
// MV_U gathers in flight instead of waiting on each column index in turn.
constexpr int MV_U = 4;
// Row kernels (row_mv) are resident MV_BLOCKS blocks per SM (64 registers a
// thread); their grids are sized to one full wave of that.
constexpr int MV_BLOCKS = 4;
// the post-smoother with column dot products (two FP64 sums per column)
constexpr int MV_BLOCKS_DOTS = 3;

// The row helpers below add to acc as the caller set it (0, or the start value
// of a folded subtraction); NEG subtracts each entry's product instead (an
// FMA with the negated value), as the single-vector kernels do.
template <int KPL, typename AccT, bool NEG = false, typename V, typename G>
__device__ __forceinline__ void row_mv(const SellView<V>& A, int64_t i, int C, int K, int lane,
                                       AccT (&acc)[KPL], G g) {
  const RowSpan r = row_span(A, i, C);
  for (int k0 = 0; k0 < r.w; k0 += MV_U) {
    int jj[MV_U];
    AccT aa[MV_U];
#pragma unroll
    for (int u = 0; u < MV_U; ++u) {
      jj[u] = 0;
      aa[u] = AccT(0);
      if (k0 + u < r.w) {
        const int64_t e = r.off + (int64_t)(k0 + u) * r.stride;
        jj[u] = __ldg(A.col + e);
        aa[u] = to_f(__ldg(A.val + e), AccT(0));
      }
    }
    AccT gg[MV_U][KPL];
#pragma unroll
    for (int u = 0; u < MV_U; ++u)
#pragma unroll
      for (int q = 0; q < KPL; ++q) {
        const int c = lane + 32 * q;
        gg[u][q] = (k0 + u < r.w && c < K) ? g(jj[u], c) : AccT(0);
      }
#pragma unroll
    for (int u = 0; u < MV_U; ++u)
      if (k0 + u < r.w)
#pragma unroll
        for (int q = 0; q < KPL; ++q) {
          const int c = lane + 32 * q;
          if (c < K) acc[q] = fma(NEG ? -aa[u] : aa[u], gg[u][q], acc[q]);
        }
  }
}

// Slices of at most SL_MAXW ELL columns and SL_CAP entries (7-point rows, and
// their A P, in slices of up to 32 rows) are staged in shared memory by the
// warp: column indices and values come in with
// coalesced loads, then every row of the slice reads its entries from there
// as broadcasts and issues all of its gathers at once, so a row costs one
// gather latency instead of a chain of index load, gather, next group.
// Entries are applied in the same order as row_mv (ELL column order, padding
// included): the results are the same bits.  Wider slices take row_mv.
// The V-cycle smoothers and the PCG product (FP32 and FP64) all walk slices
// this way.
constexpr int SL_MAXW = 8;
constexpr int SL_CAP = SL_MAXW * 32;

// Asynchronous 4- and 8-byte copies global -> shared (cp.async): the copies of a
// whole slice are in flight at once without holding registers.
template <int N>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc) {
  static_assert(N == 4 || N == 8, "4- or 8-byte copies");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(
                   (unsigned)__cvta_generic_to_shared(sdst)),
               "l"(__cvta_generic_to_global(gsrc)), "n"(N)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <typename V, typename T>
__device__ __forceinline__ bool stage_slice(const SellView<V>& A, int64_t sl, int C, int lane,
                                            int32_t* scol, T* sval, int& w) {
  const int64_t beg = __ldg(A.sliceptr + sl);
  w = (int)((__ldg(A.sliceptr + sl + 1) - beg) / C);
  if (w > SL_MAXW || w * C > SL_CAP) return false;  // slices of 64 rows fit fewer columns
  const int m = w * C;
  if constexpr (sizeof(V) == sizeof(T)) {  // values stored as computed: copied as they are
    for (int e = lane; e < m; e += 32) {
      cp_async<4>(scol + e, A.col + beg + e);
      cp_async<sizeof(T)>(sval + e, A.val + beg + e);
    }
    cp_async_wait_all();
  } else {  // BF16 values widened on the way: four entries a lane in flight per round
    for (int e0 = 0; e0 < m; e0 += 128) {
      int32_t cc[4];
      V vv[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int e = e0 + lane + 32 * k;
        if (e < m) {
          cc[k] = __ldg(A.col + beg + e);
          vv[k] = __ldg(A.val + beg + e);
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int e = e0 + lane + 32 * k;
        if (e < m) {
          scol[e] = cc[k];
          sval[e] = to_f(vv[k], T(0));
        }
      }
    }
  }
  __syncwarp();
  return true;
}

template <int KPL, bool NEG = false, typename T, typename G>
__device__ __forceinline__ void staged_row(const int32_t* scol, const T* sval, int C, int w,
                                           int r, int K, int lane, T (&acc)[KPL], G g) {
  T gg[SL_MAXW][KPL];
#pragma unroll
  for (int u = 0; u < SL_MAXW; ++u)
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
      const int c = lane + 32 * q;
      gg[u][q] = (u < w && c < K) ? g(scol[u * C + r], c) : T(0);
    }
#pragma unroll
  for (int u = 0; u < SL_MAXW; ++u)
    if (u < w) {
      const T a = NEG ? -sval[u * C + r] : sval[u * C + r];
#pragma unroll
      for (int q = 0; q < KPL; ++q)
        if (lane + 32 * q < K) acc[q] = fma(a, gg[u][q], acc[q]);
    }
}

// Two rows of a staged slice at once (the second when two): all gathers of
// both rows are in flight before either row's FMAs, so a warp waits one
// gather latency per pair of rows.
template <int KPL, bool NEG = false, typename T, typename G>
__device__ __forceinline__ void staged_rows2(const int32_t* scol, const T* sval, int C, int w,
                                             int r, bool two, int K, int lane, T (&acc0)[KPL],
                                             T (&acc1)[KPL], G g) {
  T g0[SL_MAXW][KPL], g1[SL_MAXW][KPL];
#pragma unroll
  for (int u = 0; u < SL_MAXW; ++u)
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
      const int c = lane + 32 * q;
      const bool in = u < w && c < K;
      g0[u][q] = in ? g(scol[u * C + r], c) : T(0);
      g1[u][q] = in && two ? g(scol[u * C + r + 1], c) : T(0);
    }
#pragma unroll
  for (int u = 0; u < SL_MAXW; ++u)
    if (u < w) {
      const T a0 = NEG ? -sval[u * C + r] : sval[u * C + r];
      const T a1 = two ? (NEG ? -sval[u * C + r + 1] : sval[u * C + r + 1]) : T(0);
#pragma unroll
      for (int q = 0; q < KPL; ++q)
        if (lane + 32 * q < K) {
          acc0[q] = fma(a0, g0[u][q], acc0[q]);
          acc1[q] = fma(a1, g1[u][q], acc1[q]);
        }
    }
}

// Column sums over the grid: per-block sums in fixed warp order, then the
// last block adds the blocks in order and calls epi(c, t) for every column.
// sh[m][w][c]: warp w's sum of value m for column c.
template <int NV, typename Epi>
__device__ void cols_finish(double (&sh)[NV][MROWS_BLOCK / 32][64], int K, double* part,
                            int maxb, unsigned* ticket, Epi epi) {
  __shared__ bool last;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int t = threadIdx.x; t < NV * K; t += blockDim.x) {
    const int m = t / K, c = t % K;
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += sh[m][k][c];
    part[((size_t)m * maxb + blockIdx.x) * K + c] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // the last block: thread t adds every G-th block's partial of column t % K
  // starting at block t / K (G = blockDim / K groups), then thread c < K adds
  // the G group sums in order -- fixed assignment, fixed order
  __shared__ double gs[NV][MROWS_BLOCK];
  const int G = blockDim.x / K;
  const int c0 = threadIdx.x % K, g0 = threadIdx.x / K;
  double t0[NV];
#pragma unroll
  for (int m = 0; m < NV; ++m) t0[m] = 0.0;
  if (g0 < G)
#pragma unroll 8
    for (int b = g0; b < (int)gridDim.x; b += G)
#pragma unroll
      for (int m = 0; m < NV; ++m) t0[m] += __ldcg(&part[((size_t)m * maxb + b) * K + c0]);
#pragma unroll
  for (int m = 0; m < NV; ++m) gs[m][threadIdx.x] = t0[m];
  __syncthreads();
  if (threadIdx.x < K) {
    double t[NV];
#pragma unroll
    for (int m = 0; m < NV; ++m) {
      double s = 0.0;
      for (int g = 0; g < G; ++g) s += gs[m][g * K + threadIdx.x];
      t[m] = s;
    }
    epi(threadIdx.x, t);
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// Lane l holds columns l + 32 q.
template <int KPL, int NV, typename Epi>
__device__ void cols_reduce(double (&v)[NV][KPL], int K, double* part, int maxb,
                            unsigned* ticket, Epi epi) {
  __shared__ double sh[NV][MROWS_BLOCK / 32][64];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int m = 0; m < NV; ++m)
#pragma unroll
    for (int q = 0; q < KPL; ++q) sh[m][w][lane + 32 * q] = v[m][q];
  cols_finish(sh, K, part, maxb, ticket, epi);
}

// Vector-column lanes (see k_m_pre_v): lane (rs, cg) holds columns
// cg VW .. cg VW + VW - 1 of the rows it took; the warp's RW row lanes of a
// column are added in row-lane order.
template <int VW, int NV, typename Epi>
__device__ void cols_reduce_v(double (&v)[NV][VW], int K, double* part, int maxb,
                              unsigned* ticket, Epi epi) {
  __shared__ double sh[NV][MROWS_BLOCK / 32][64];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int G = K / VW, RW = 32 / G, cg = lane % G, rs = lane / G;
  for (int k = 0; k < RW; ++k) {
    if (rs == k)
#pragma unroll
      for (int m = 0; m < NV; ++m)
#pragma unroll
        for (int j = 0; j < VW; ++j) {
          double& t = sh[m][w][cg * VW + j];
          t = k == 0 ? v[m][j] : t + v[m][j];
        }
    __syncwarp();
  }
  cols_finish(sh, K, part, maxb, ticket, epi);
}

// ------------------------------------------------------------------ V-cycle kernels

// One warp per slice (staged slices, see stage_slice).
template <int KPL, typename V, typename T, typename BT>
__global__ void __launch_bounds__(MROWS_BLOCK, MV_BLOCKS)
    k_m_pre(SellView<V> Ah, int C, int K, const BT* __restrict__ B, T* __restrict__ R) {
  __shared__ int32_t scol_all[MROWS_BLOCK / 32][SL_CAP];
  __shared__ T sval_all[MROWS_BLOCK / 32][SL_CAP];
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t* scol = scol_all[threadIdx.x >> 5];
  T* sval = sval_all[threadIdx.x >> 5];
  auto gather = [&](int j, int c) { return to_f(__ldg(B + (int64_t)j * K + c), T(0)); };
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < Ah.nslices;
       sl += nw) {
    const int64_t i0 = sl * C;
    const int rows = (int)(Ah.n - i0 < C ? Ah.n - i0 : C);
    int w;
    const bool staged = stage_slice(Ah, sl, C, lane, scol, sval, w);
    // r = b - Ah b as the single-vector kernels form it: from b down by
    // negated FMAs
    auto start = [&](int64_t i, T(&acc)[KPL]) {
#pragma unroll
      for (int q = 0; q < KPL; ++q) {
        const int c = lane + 32 * q;
        acc[q] = c < K ? to_f(B[i * K + c], T(0)) : T(0);
      }
    };
    auto finish = [&](int64_t i, const T(&acc)[KPL]) {
#pragma unroll
      for (int q = 0; q < KPL; ++q) {
        const int c = lane + 32 * q;
        if (c < K) R[i * K + c] = acc[q];
      }
    };
    // FP32 vectors: two rows in flight; FP64 ones (twice the registers): one
    constexpr int RS = sizeof(T) == 4 ? 2 : 1;
    for (int r = 0; r < rows; r += RS) {
      const bool two = RS == 2 && r + 1 < rows;
      T acc0[KPL], acc1[KPL];
      start(i0 + r, acc0);
      if (two) start(i0 + r + 1, acc1);
      if (staged && RS == 2) {
        staged_rows2<KPL, true>(scol, sval, C, w, r, two, K, lane, acc0, acc1, gather);
      } else if (staged) {
        staged_row<KPL, true>(scol, sval, C, w, r, K, lane, acc0, gather);
      } else {
        row_mv<KPL, T, true>(Ah, i0 + r, C, K, lane, acc0, gather);
        if (two) row_mv<KPL, T, true>(Ah, i0 + r + 1, C, K, lane, acc1, gather);
      }
      finish(i0 + r, acc0);
      if (two) finish(i0 + r + 1, acc1);
    }
    __syncwarp();  // the next slice overwrites the staging
  }
}

// w = v rounded to FP32, four elements a thread (16-byte loads when v and w
// are 16-byte aligned, vec = true).
__global__ void k_m_to_f32(int64_t m, const double* __restrict__ v, float* __restrict__ w,
                           bool vec) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * t < m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = 4 * t;
    double a[4];
    float b[4];
    if (vec && i + 4 <= m) {
      const double2 a0 = __ldcs((const double2*)(v + i)), a1 = __ldcs((const double2*)(v + i + 2));
      a[0] = a0.x, a[1] = a0.y, a[2] = a1.x, a[3] = a1.y;
      cvt_n(a, b);
      *(float4*)(w + i) = make_float4(b[0], b[1], b[2], b[3]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = i + k < m ? v[i + k] : 0.0;
      cvt_n(a, b);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (i + k < m) w[i + k] = b[k];
    }
  }
}

template <typename T>
__global__ void k_m_restrict(int64_t nc, int stride, int K, const int32_t* __restrict__ members,
                             const T* __restrict__ R, T* __restrict__ Bc) {
  const int64_t total = nc * K;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = t / K;
    const int c = (int)(t % K);
    const int32_t* m = members + I * stride;
    T acc = R[(int64_t)m[0] * K + c];
    for (int k = 1; k < stride; ++k) {
      const int32_t i = m[k];
      if (i < 0) break;
      acc = acc + R[(int64_t)i * K + c];
    }
    Bc[t] = acc;
  }
}

struct MultiRzEpi {
  Scal* sc;
  int beta_form;
  int first;
  __device__ void operator()(int c, const double (&t)[2]) const {
    Scal& S = sc[c];
    if (first) {
      S.rz = t[0];
      return;
    }
    if (!S.active) return;
    S.beta = beta_form == PCG_BETA_FLEXIBLE ? -t[1] / S.pq : t[0] / S.rz;
    S.zq = t[1];
    S.rz = t[0];
    if (!isfinite(t[0])) {
      S.status = AMG_ERR_NAN;
      S.active = 0;
    }
  }
};

template <int KPL, typename V, typename T, typename BT, typename XT, bool DOTS>
__global__ void __launch_bounds__(MROWS_BLOCK, MV_BLOCKS)
    k_m_post(SellView<V> AP, int C, int K, const BT* __restrict__ B, const T* __restrict__ s,
             const T* __restrict__ R, const int32_t* __restrict__ agg, const T* __restrict__ Xc,
             XT* __restrict__ Z, const double* __restrict__ Q, double* part, int maxb,
             unsigned* ticket, MultiRzEpi epi) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double d[2][KPL];
#pragma unroll
  for (int q = 0; q < KPL; ++q) d[0][q] = d[1][q] = 0.0;
  __shared__ int32_t scol_all[MROWS_BLOCK / 32][SL_CAP];
  __shared__ T sval_all[MROWS_BLOCK / 32][SL_CAP];
  int32_t* scol = scol_all[threadIdx.x >> 5];
  T* sval = sval_all[threadIdx.x >> 5];
  auto gather = [&](int J, int c) { return __ldg(Xc + (int64_t)J * K + c); };
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < AP.nslices;
       sl += nw) {
    const int64_t i0 = sl * C;
    const int rows = (int)(AP.n - i0 < C ? AP.n - i0 : C);
    int w;
    const bool staged = stage_slice(AP, sl, C, lane, scol, sval, w);
    // z = s (b + r - AP x_c) + x_c[agg] as the single-vector kernels form it:
    // from b + r down by negated FMAs, then one FMA
    auto start = [&](int64_t i, T(&acc)[KPL]) {
      BT bv[KPL];
      T rr[KPL];
#pragma unroll
      for (int q = 0; q < KPL; ++q) {
        const int c = lane + 32 * q;
        bv[q] = c < K ? B[i * K + c] : BT(0);
        rr[q] = c < K ? R[i * K + c] : T(0);
      }
      cvt_n(bv, acc);
#pragma unroll
      for (int q = 0; q < KPL; ++q) acc[q] = acc[q] + rr[q];
    };
    auto finish = [&](int64_t i, const T(&acc)[KPL]) {
      const T si = s[i];
      const int64_t ai = agg[i];
      T zt[KPL];
#pragma unroll
      for (int q = 0; q < KPL; ++q) {
        const int c = lane + 32 * q;
        zt[q] = c < K ? fma(si, acc[q], Xc[ai * K + c]) : T(0);
      }
      XT zv[KPL];
      cvt_n(zt, zv);
#pragma unroll
      for (int q = 0; q < KPL; ++q) {
        const int c = lane + 32 * q;
        if (c < K) {
          Z[i * K + c] = zv[q];
          if (DOTS) {
            d[0][q] += (double)B[i * K + c] * (double)zv[q];
            d[1][q] += (double)zv[q] * Q[i * K + c];
          }
        }
      }
    };
    // FP32 vectors: two rows in flight; FP64 ones (twice the registers): one
    constexpr int RS = sizeof(T) == 4 ? 2 : 1;
    for (int r = 0; r < rows; r += RS) {
      const bool two = RS == 2 && r + 1 < rows;
      T acc0[KPL], acc1[KPL];
      start(i0 + r, acc0);
      if (two) start(i0 + r + 1, acc1);
      if (staged && RS == 2) {
        staged_rows2<KPL, true>(scol, sval, C, w, r, two, K, lane, acc0, acc1, gather);
      } else if (staged) {
        staged_row<KPL, true>(scol, sval, C, w, r, K, lane, acc0, gather);
      } else {
        row_mv<KPL, T, true>(AP, i0 + r, C, K, lane, acc0, gather);
        if (two) row_mv<KPL, T, true>(AP, i0 + r + 1, C, K, lane, acc1, gather);
      }
      finish(i0 + r, acc0);
      if (two) finish(i0 + r + 1, acc1);
    }
    __syncwarp();
  }
  if constexpr (DOTS) cols_reduce<KPL, 2>(d, K, part, maxb, ticket, epi);
}

// ------------------------------------------------------------------ vector-column kernels
//
// The smoothers again, with each lane on VW = 16 / sizeof(T) adjacent columns
// of one row (one 16-byte access per gathered row) instead of on columns
// l and l + 32: lane l takes column group cg = l % G (G = K / VW groups) of
// row rs = l / G of the RW = 32 / G rows a warp advances by per pass (lanes
// past RW G idle).  A warp's gather then moves RW rows' K values in one
// instruction, where the per-column kernels spend K / 32 instructions on one
// row, so the slices' rows cost a fraction of the issue slots.  Per element the
// arithmetic and its order are unchanged (start value, then one negated FMA
// per ELL entry, padding included, then the final FMA), so the results are the
// single-vector V-cycle's bits.  Used when VW divides K and every vector
// starts on 16 bytes.

template <int N>
__device__ __forceinline__ void ld_cols(const float* __restrict__ p, float (&o)[N]) {
  static_assert(N % 4 == 0, "four floats per access");
#pragma unroll
  for (int k = 0; k < N / 4; ++k) {
    const float4 v = __ldg((const float4*)p + k);
    o[4 * k] = v.x, o[4 * k + 1] = v.y, o[4 * k + 2] = v.z, o[4 * k + 3] = v.w;
  }
}
template <int N>
__device__ __forceinline__ void ld_cols(const double* __restrict__ p, double (&o)[N]) {
  static_assert(N % 2 == 0, "two doubles per access");
#pragma unroll
  for (int k = 0; k < N / 2; ++k) {
    const double2 v = __ldg((const double2*)p + k);
    o[2 * k] = v.x, o[2 * k + 1] = v.y;
  }
}
template <int N>
__device__ __forceinline__ void st_cols(float* __restrict__ p, const float (&o)[N]) {
#pragma unroll
  for (int k = 0; k < N / 4; ++k)
    ((float4*)p)[k] = make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
}
template <int N>
__device__ __forceinline__ void st_cols(double* __restrict__ p, const double (&o)[N]) {
#pragma unroll
  for (int k = 0; k < N / 2; ++k) ((double2*)p)[k] = make_double2(o[2 * k], o[2 * k + 1]);
}

// acc -= sum_k a_ik X[col_k, c0 ..] for the lane's row (staged slice, or the
// row's entries from global memory when the slice did not fit the staging);
// acc += ... with NEG false.
template <int VW, bool NEG = true, typename V, typename T>
__device__ __forceinline__ void rows_sub_v(const SellView<V>& A, bool staged, const int32_t* scol,
                                           const T* sval, int C, int w, int r, int64_t i, int K,
                                           int c0, const T* __restrict__ X, T (&acc)[VW]) {
  if (staged) {
    T g[SL_MAXW][VW];
#pragma unroll
    for (int u = 0; u < SL_MAXW; ++u) {
      if (u < w) {
        ld_cols(X + (int64_t)scol[u * C + r] * K + c0, g[u]);
      } else {
#pragma unroll
        for (int k = 0; k < VW; ++k) g[u][k] = T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < SL_MAXW; ++u)
      if (u < w) {
        const T a = NEG ? -sval[u * C + r] : sval[u * C + r];
#pragma unroll
        for (int k = 0; k < VW; ++k) acc[k] = fma(a, g[u][k], acc[k]);
      }
    return;
  }
  const RowSpan rw = row_span(A, i, C);
  for (int k0 = 0; k0 < rw.w; k0 += MV_U) {
    int jj[MV_U];
    T aa[MV_U];
    T g[MV_U][VW];
#pragma unroll
    for (int u = 0; u < MV_U; ++u) {
      jj[u] = 0;
      aa[u] = T(0);
      if (k0 + u < rw.w) {
        const int64_t e = rw.off + (int64_t)(k0 + u) * rw.stride;
        jj[u] = __ldg(A.col + e);
        aa[u] = to_f(__ldg(A.val + e), T(0));
      }
    }
#pragma unroll
    for (int u = 0; u < MV_U; ++u) {
      if (k0 + u < rw.w) {
        ld_cols(X + (int64_t)jj[u] * K + c0, g[u]);
      } else {
#pragma unroll
        for (int k = 0; k < VW; ++k) g[u][k] = T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < MV_U; ++u)
      if (k0 + u < rw.w)
#pragma unroll
        for (int k = 0; k < VW; ++k) acc[k] = fma(NEG ? -aa[u] : aa[u], g[u][k], acc[k]);
  }
}

// R = B - Ah B (as k_m_pre), vector columns.
template <typename V, typename T>
__global__ void __launch_bounds__(MROWS_BLOCK, MV_BLOCKS)
    k_m_pre_v(SellView<V> Ah, int C, int K, const T* __restrict__ B, T* __restrict__ R) {
  constexpr int VW = 16 / sizeof(T);
  __shared__ int32_t scol_all[MROWS_BLOCK / 32][SL_CAP];
  __shared__ T sval_all[MROWS_BLOCK / 32][SL_CAP];
  const int lane = threadIdx.x & 31;
  const int G = K / VW, RW = 32 / G, cg = lane % G, rs = lane / G, c0 = cg * VW;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t* scol = scol_all[threadIdx.x >> 5];
  T* sval = sval_all[threadIdx.x >> 5];
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < Ah.nslices;
       sl += nw) {
    const int64_t i0 = sl * C;
    const int rows = (int)(Ah.n - i0 < C ? Ah.n - i0 : C);
    int w;
    const bool staged = stage_slice(Ah, sl, C, lane, scol, sval, w);
    for (int p = 0; p < rows; p += RW) {
      const bool live = rs < RW && p + rs < rows;
      const int r = live ? p + rs : 0;  // idle lanes shadow row 0 and store nothing
      const int64_t i = i0 + r;
      T acc[VW];
      ld_cols(B + i * K + c0, acc);
      rows_sub_v<VW>(Ah, staged, scol, sval, C, w, r, i, K, c0, B, acc);
      if (live) st_cols(R + i * K + c0, acc);
    }
    __syncwarp();  // the next slice overwrites the staging
  }
}

// Z = s (B + R - AP Xc) + Xc[agg] (as k_m_post), vector columns; with DOTS
// the column sums (B, Z) and (Z, Q) go to epi.
template <typename V, typename T, typename BT, typename XT, bool DOTS>
__global__ void __launch_bounds__(MROWS_BLOCK, DOTS ? MV_BLOCKS_DOTS : MV_BLOCKS)
    k_m_post_v(SellView<V> AP, int C, int K, const BT* __restrict__ B, const T* __restrict__ s,
               const T* __restrict__ R, const int32_t* __restrict__ agg,
               const T* __restrict__ Xc, XT* __restrict__ Z, const double* __restrict__ Q,
               double* part, int maxb, unsigned* ticket, MultiRzEpi epi) {
  constexpr int VW = 16 / sizeof(T);
  __shared__ int32_t scol_all[MROWS_BLOCK / 32][SL_CAP];
  __shared__ T sval_all[MROWS_BLOCK / 32][SL_CAP];
  const int lane = threadIdx.x & 31;
  const int G = K / VW, RW = 32 / G, cg = lane % G, rs = lane / G, c0 = cg * VW;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t* scol = scol_all[threadIdx.x >> 5];
  T* sval = sval_all[threadIdx.x >> 5];
  double d[2][VW];
#pragma unroll
  for (int k = 0; k < VW; ++k) d[0][k] = d[1][k] = 0.0;
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < AP.nslices;
       sl += nw) {
    const int64_t i0 = sl * C;
    const int rows = (int)(AP.n - i0 < C ? AP.n - i0 : C);
    int w;
    const bool staged = stage_slice(AP, sl, C, lane, scol, sval, w);
    for (int p = 0; p < rows; p += RW) {
      const bool live = rs < RW && p + rs < rows;
      const int r = live ? p + rs : 0;
      const int64_t i = i0 + r;
      T acc[VW];
      {
        BT bv[VW];
        T rv[VW];
        ld_cols(B + i * K + c0, bv);
        ld_cols(R + i * K + c0, rv);
        cvt_n(bv, acc);
#pragma unroll
        for (int k = 0; k < VW; ++k) acc[k] = acc[k] + rv[k];
      }
      rows_sub_v<VW>(AP, staged, scol, sval, C, w, r, i, K, c0, Xc, acc);
      const T si = s[i];
      T xv[VW];
      ld_cols(Xc + (int64_t)agg[i] * K + c0, xv);
#pragma unroll
      for (int k = 0; k < VW; ++k) xv[k] = fma(si, acc[k], xv[k]);
      XT zv[VW];
      cvt_n(xv, zv);
      if (live) {
        st_cols(Z + i * K + c0, zv);
        if constexpr (DOTS) {
          BT bv[VW];
          double qv[VW];
          ld_cols(B + i * K + c0, bv);
          ld_cols(Q + i * K + c0, qv);
#pragma unroll
          for (int k = 0; k < VW; ++k) {
            d[0][k] += (double)bv[k] * (double)zv[k];
            d[1][k] += (double)zv[k] * qv[k];
          }
        }
      }
    }
    __syncwarp();
  }
  if constexpr (DOTS) cols_reduce_v<VW, 2>(d, K, part, maxb, ticket, epi);
}

// Restriction with vector columns: thread t sums column group t % G (VW
// columns, G = K / VW) of aggregate t / G.  The member indices come first,
// then all their rows' loads, then the additions in member order (as
// k_m_restrict adds them; the list ends at the first negative index).
constexpr int RS_U = 8;
template <typename T>
__global__ void k_m_restrict_v(int64_t nc, int stride, int K,
                               const int32_t* __restrict__ members, const T* __restrict__ R,
                               T* __restrict__ Bc) {
  constexpr int VW = 16 / sizeof(T);
  const int G = K / VW;
  const int64_t total = nc * G;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t I = t / G;
    const int c0 = (int)(t % G) * VW;
    const int32_t* m = members + I * stride;
    T acc[VW];
    ld_cols(R + (int64_t)__ldg(m) * K + c0, acc);
    bool live = true;
    for (int k0 = 1; k0 < stride && live; k0 += RS_U) {
      int ii[RS_U];
#pragma unroll
      for (int u = 0; u < RS_U; ++u) ii[u] = k0 + u < stride ? __ldg(m + k0 + u) : -1;
      T g[RS_U][VW];
#pragma unroll
      for (int u = 0; u < RS_U; ++u) {
        if (ii[u] >= 0) {
          ld_cols(R + (int64_t)ii[u] * K + c0, g[u]);
        } else {
#pragma unroll
          for (int k = 0; k < VW; ++k) g[u][k] = T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < RS_U; ++u) {
        live = live && ii[u] >= 0;
        if (live)
#pragma unroll
          for (int k = 0; k < VW; ++k) acc[k] = acc[k] + g[u][k];
      }
    }
    st_cols(Bc + I * K + c0, acc);
  }
}

// Coarsest level for K columns: Y = L^-1 B, then X = L^-T Y, one thread per
// output element (n <= 3072).  Each dot product is summed exactly as the
// single-RHS coarse kernel sums it: 32 lane partials over a stride of 32,
// combined by the same xor-butterfly tree.
__device__ __forceinline__ double lane_tree(double (&p)[32]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int l = 0; l < o; ++l) p[l] = p[l] + p[l + o];
  return p[0];
}

template <typename BT>
__global__ void k_m_coarse1(int64_t n, int K, int nblk, const int64_t* __restrict__ brow,
                            const int64_t* __restrict__ bmat, const double* __restrict__ Linv,
                            const BT* __restrict__ B, double* __restrict__ Y) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * K;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gi = t / K;
    const int c = (int)(t % K);
    const int b = coarse_block(brow, nblk, gi);
    const int64_t r0 = brow[b];
    const int m = (int)(brow[b + 1] - r0), i = (int)(gi - r0);
    const double* L = Linv + bmat[b];
    double p[32];
#pragma unroll
    for (int l = 0; l < 32; ++l) p[l] = 0.0;
    for (int k = 0; k <= i; ++k)
      p[k & 31] = fma(L[(int64_t)i * m + k], (double)B[(r0 + k) * K + c], p[k & 31]);
    Y[t] = lane_tree(p);
  }
}

template <typename XT>
__global__ void k_m_coarse2(int64_t n, int K, int nblk, const int64_t* __restrict__ brow,
                            const int64_t* __restrict__ bmat, const double* __restrict__ LinvT,
                            const double* __restrict__ Y, XT* __restrict__ X) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * K;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gk = t / K;
    const int c = (int)(t % K);
    const int b = coarse_block(brow, nblk, gk);
    const int64_t r0 = brow[b];
    const int m = (int)(brow[b + 1] - r0), k = (int)(gk - r0);
    const double* LT = LinvT + bmat[b];
    double p[32];
#pragma unroll
    for (int l = 0; l < 32; ++l) p[l] = 0.0;
    for (int i = k; i < m; ++i)
      p[(i - k) & 31] = fma(LT[(int64_t)k * m + i], Y[(r0 + i) * K + c], p[(i - k) & 31]);
    X[t] = (XT)lane_tree(p);
  }
}

// ------------------------------------------------------------------ PCG kernels

struct MultiInitEpi {
  Scal* sc;
  double tol;
  int maxit;
  int* nactive;
  int mode;  // 0: initial residual, 1: true residual at exit
  __device__ void operator()(int c, const double (&t)[2]) const {
    Scal& S = sc[c];
    if (mode == 1) {
      S.tr = t[0];
      return;
    }
    S.rr = t[0];
    S.bb = t[1];
    S.iters = 0;
    S.pq_fail = 0;
    const double bn = t[1] > 0.0 ? sqrt(t[1]) : 1.0;
    const bool done = sqrt(t[0]) / bn <= tol;
    S.status = done ? AMG_OK : AMG_NOT_CONVERGED;
    S.active = (!done && maxit > 0) ? 1 : 0;
    if (S.active) atomicAdd(nactive, 1);
  }
};

template <int KPL>
__global__ void __launch_bounds__(MROWS_BLOCK, MV_BLOCKS)
    k_m_residual(SellView<double> A, int C, int K, const double* __restrict__ B,
                 const double* __restrict__ X, double* __restrict__ R, double* part, int maxb,
                 unsigned* ticket, MultiInitEpi epi, float* __restrict__ R32) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double d[2][KPL];
#pragma unroll
  for (int q = 0; q < KPL; ++q) d[0][q] = d[1][q] = 0.0;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < A.n; i += nw) {
    double acc[KPL];
#pragma unroll
    for (int q = 0; q < KPL; ++q) acc[q] = 0.0;
    row_mv<KPL, double>(A, i, C, K, lane, acc,
                        [&](int j, int c) { return __ldg(X + (int64_t)j * K + c); });
    double rv[KPL];
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
      const int c = lane + 32 * q;
      rv[q] = 0.0;
      if (c < K) {
        const double bi = B[i * K + c];
        const double ri = bi - acc[q];
        rv[q] = ri;
        R[i * K + c] = ri;
        d[0][q] += ri * ri;
        d[1][q] += bi * bi;
      }
    }
    if (R32) {
      float r32[KPL];
      cvt_n(rv, r32);
#pragma unroll
      for (int q = 0; q < KPL; ++q)
        if (lane + 32 * q < K) R32[i * K + lane + 32 * q] = r32[q];
    }
  }
  cols_reduce<KPL, 2>(d, K, part, maxb, ticket, epi);
}

struct MultiPqEpi {
  Scal* sc;
  __device__ void operator()(int c, const double (&t)[1]) const {
    Scal& S = sc[c];
    if (!S.active) {
      S.alpha = 0.0;
      return;
    }
    S.pq = t[0];
    S.alpha = S.rz / t[0];
    if (!(t[0] > 0.0)) {
      S.status = isfinite(t[0]) ? AMG_ERR_BREAKDOWN : AMG_ERR_NAN;
      S.pq_fail = 1;
      S.active = 0;
      S.alpha = 0.0;
    }
  }
};

template <int KPL>
__global__ void __launch_bounds__(MROWS_BLOCK, MV_BLOCKS)
    k_m_spmm_dot(SellView<double> A, int C, int K, const double* __restrict__ P,
                 double* __restrict__ Q, double* part, int maxb, unsigned* ticket, MultiPqEpi epi) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double d[1][KPL];
#pragma unroll
  for (int q = 0; q < KPL; ++q) d[0][q] = 0.0;
  __shared__ int32_t scol_all[MROWS_BLOCK / 32][SL_CAP];
  __shared__ double sval_all[MROWS_BLOCK / 32][SL_CAP];
  int32_t* scol = scol_all[threadIdx.x >> 5];
  double* sval = sval_all[threadIdx.x >> 5];
  auto gather = [&](int j, int c) { return __ldg(P + (int64_t)j * K + c); };
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < A.nslices;
       sl += nw) {
    const int64_t i0 = sl * C;
    const int rows = (int)(A.n - i0 < C ? A.n - i0 : C);
    int w;
    const bool staged = stage_slice(A, sl, C, lane, scol, sval, w);
    for (int r = 0; r < rows; ++r) {
      const int64_t i = i0 + r;
      double acc[KPL];
#pragma unroll
      for (int q = 0; q < KPL; ++q) acc[q] = 0.0;
      if (staged)
        staged_row<KPL>(scol, sval, C, w, r, K, lane, acc, gather);
      else
        row_mv<KPL, double>(A, i, C, K, lane, acc, gather);
#pragma unroll
      for (int q = 0; q < KPL; ++q) {
        const int c = lane + 32 * q;
        if (c < K) {
          Q[i * K + c] = acc[q];
          d[0][q] += P[i * K + c] * acc[q];
        }
      }
    }
    __syncwarp();
  }
  cols_reduce<KPL, 1>(d, K, part, maxb, ticket, epi);
}

// Q = A P and (p, q) per column, vector columns (two doubles a lane); see
// k_m_pre_v for the lane layout.
__global__ void __launch_bounds__(MROWS_BLOCK, MV_BLOCKS)
    k_m_spmm_dot_v(SellView<double> A, int C, int K, const double* __restrict__ P,
                   double* __restrict__ Q, double* part, int maxb, unsigned* ticket,
                   MultiPqEpi epi) {
  constexpr int VW = 2;
  __shared__ int32_t scol_all[MROWS_BLOCK / 32][SL_CAP];
  __shared__ double sval_all[MROWS_BLOCK / 32][SL_CAP];
  const int lane = threadIdx.x & 31;
  const int G = K / VW, RW = 32 / G, cg = lane % G, rs = lane / G, c0 = cg * VW;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int32_t* scol = scol_all[threadIdx.x >> 5];
  double* sval = sval_all[threadIdx.x >> 5];
  double d[1][VW] = {{0.0, 0.0}};
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < A.nslices;
       sl += nw) {
    const int64_t i0 = sl * C;
    const int rows = (int)(A.n - i0 < C ? A.n - i0 : C);
    int w;
    const bool staged = stage_slice(A, sl, C, lane, scol, sval, w);
    for (int p = 0; p < rows; p += RW) {
      const bool live = rs < RW && p + rs < rows;
      const int r = live ? p + rs : 0;
      const int64_t i = i0 + r;
      double acc[VW] = {0.0, 0.0};
      rows_sub_v<VW, false>(A, staged, scol, sval, C, w, r, i, K, c0, P, acc);
      if (live) {
        st_cols(Q + i * K + c0, acc);
        double pv[VW];
        ld_cols(P + i * K + c0, pv);
#pragma unroll
        for (int k = 0; k < VW; ++k) d[0][k] += pv[k] * acc[k];
      }
    }
    __syncwarp();
  }
  cols_reduce_v<VW, 1>(d, K, part, maxb, ticket, epi);
}

struct MultiRrEpi {
  Scal* sc;
  double tol;
  int maxit;
  int* nactive;
  __device__ void operator()(int c, const double (&t)[1]) const {
    Scal& S = sc[c];
    if (!S.active) return;
    S.rr = t[0];
    S.iters += 1;
    const double bn = S.bb > 0.0 ? sqrt(S.bb) : 1.0;
    const double rel = sqrt(t[0]) / bn;
    if (!isfinite(t[0])) {
      S.status = AMG_ERR_NAN;
      S.active = 0;
    } else if (rel <= tol) {
      S.status = AMG_OK;
      S.active = 0;
    } else if (S.iters >= maxit) {
      S.status = AMG_NOT_CONVERGED;
      S.active = 0;
    }
    if (S.active) atomicAdd(nactive, 1);
  }
};

// x += alpha_c p; r -= alpha_c q; (r, r) per column (alpha_c = 0 when frozen).
template <int KPL>
__global__ void __launch_bounds__(MROWS_BLOCK)
    k_m_update(int64_t n, int K, double* __restrict__ X, double* __restrict__ R,
               const double* __restrict__ P, const double* __restrict__ Q, const Scal* sc,
               double* part, int maxb, unsigned* ticket, MultiRrEpi epi,
               float* __restrict__ R32) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double al[KPL], d[1][KPL];
  bool act[KPL];
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int c = lane + 32 * q;
    act[q] = c < K && sc[c].active;
    al[q] = act[q] ? sc[c].alpha : 0.0;
    d[0][q] = 0.0;
  }
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    double rv[KPL];
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
      const int c = lane + 32 * q;
      rv[q] = 0.0;
      if (act[q]) {
        const int64_t e = i * K + c;
        X[e] = X[e] + al[q] * P[e];
        const double ri = R[e] - al[q] * Q[e];
        rv[q] = ri;
        R[e] = ri;
        d[0][q] += ri * ri;
      }
    }
    if (R32) {
      float r32[KPL];
      cvt_n(rv, r32);
#pragma unroll
      for (int q = 0; q < KPL; ++q)
        if (act[q]) R32[i * K + lane + 32 * q] = r32[q];
    }
  }
  cols_reduce<KPL, 1>(d, K, part, maxb, ticket, epi);
}

// p = z + beta_c p for columns still iterating.
template <int KPL>
__global__ void k_m_p_update(int64_t n, int K, double* __restrict__ P, const double* __restrict__ Z,
                             const Scal* sc) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double be[KPL];
  bool act[KPL];
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int c = lane + 32 * q;
    act[q] = c < K && sc[c].active;
    be[q] = act[q] ? sc[c].beta : 0.0;
  }
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw)
#pragma unroll
    for (int q = 0; q < KPL; ++q)
      if (act[q]) {
        const int64_t e = i * K + lane + 32 * q;
        P[e] = Z[e] + be[q] * P[e];
      }
}

// ------------------------------------------------------------------ driver

#define AMG_DISPATCH_KPL(K, ...)          \
  if ((K) <= 32) {                        \
    constexpr int KPL = 1;                \
    __VA_ARGS__;                          \
  } else {                                \
    constexpr int KPL = 2;                \
    __VA_ARGS__;                          \
  }

static int mgrid(const amg_handle* H, int64_t rows) {
  return grid_for(rows * 32, MROWS_BLOCK, H->num_sms, 8);
}
static int mgrid_mv(const amg_handle* H, int64_t rows) {
  return grid_for(rows * 32, MROWS_BLOCK, H->num_sms, MV_BLOCKS);
}

// Smoother launches: the vector-column kernels when vec (VW divides K, all
// vectors 16-byte aligned), else the per-column ones.
template <typename V, typename T>
static void m_pre(const amg_handle* H, bool vec, int K, const Level& L, const SellView<V>& v,
                  const T* b, T* r, cudaStream_t s) {
  const int g = mgrid_mv(H, L.n);
  if (vec)
    k_m_pre_v<V, T><<<g, MROWS_BLOCK, 0, s>>>(v, L.A.C, K, b, r);
  else
    AMG_DISPATCH_KPL(K, (k_m_pre<KPL, V, T, T><<<g, MROWS_BLOCK, 0, s>>>(v, L.A.C, K, b, r)));
}

template <bool DOTS, typename V, typename T, typename BT, typename XT>
static void m_post(const amg_handle* H, const MultiWs& W, bool vec, int K, const Level& L,
                   const SellView<V>& v, const BT* b, const T* xc, XT* z, const double* Q,
                   MultiRzEpi epi, cudaStream_t s) {
  const T* sv = (const T*)(sizeof(T) == 8 ? (const void*)L.s64 : (const void*)L.s32);
  const T* rv = (const T*)W.lr[&L - H->L.data()];
  const int maxb = H->red.max_blocks;
  if (vec) {
    const int g = grid_for(L.n * 32, MROWS_BLOCK, H->num_sms, DOTS ? MV_BLOCKS_DOTS : MV_BLOCKS);
    k_m_post_v<V, T, BT, XT, DOTS><<<g, MROWS_BLOCK, 0, s>>>(
        v, L.AP.C, K, b, sv, rv, L.agg, xc, z, Q, W.part, maxb, W.ticket, epi);
  } else {
    const int g = mgrid_mv(H, L.n);
    AMG_DISPATCH_KPL(K, (k_m_post<KPL, V, T, BT, XT, DOTS><<<g, MROWS_BLOCK, 0, s>>>(
                            v, L.AP.C, K, b, sv, rv, L.agg, xc, z, Q, W.part, maxb, W.ticket,
                            epi)));
  }
}

// R32: the FP32 copy of R0 (FP32 hierarchies), read by the level-0
// pre-smoother: each element is converted once, not once per gather.
template <typename T>
static int m_vcycle(const amg_handle* H, const MultiWs& W, const double* R0, double* Z0,
                    bool dots, const double* Q, int beta_form, bool first, cudaStream_t s,
                    const float* R32) {
  const int K = W.K;
  const int nl = (int)H->L.size();
  MultiRzEpi epi{W.sc, beta_form, first ? 1 : 0};
  auto coarse = [&](const auto* b, auto* x) -> int {
    const int64_t n = H->nco;
    const int g = grid_for(n * K, 256, H->num_sms, 4);
    k_m_coarse1<<<g, 256, 0, s>>>(n, K, H->nblk, H->d_brow, H->d_bmat, H->Linv, b, W.cy);
    AMG_LAUNCH_CHECK();
    k_m_coarse2<<<g, 256, 0, s>>>(n, K, H->nblk, H->d_brow, H->d_bmat, H->LinvT, W.cy, x);
    AMG_LAUNCH_CHECK();
    return AMG_OK;
  };
  if (nl == 1) return AMG_ERR_UNSUPPORTED;  // single-level hierarchies: use pcg_solve
  if (sizeof(T) == 4 && !R32) return AMG_ERR_ARG;
  // the workspace is 256-byte aligned; R0, Z0 (and R32, Q) are checked
  const bool vec = K % (16 / (int)sizeof(T)) == 0 &&
                   (((uintptr_t)R0 | (uintptr_t)Z0 | (uintptr_t)R32 | (uintptr_t)Q) & 15u) == 0;
  for (int l = 0; l < nl - 1; ++l) {
    const Level& L = H->L[l];
    T* r = (T*)W.lr[l];
    if constexpr (sizeof(T) == 8) {
      m_pre(H, vec, K, L, view<double>(L.A, L.ah64), l == 0 ? R0 : (const double*)W.lb[l], r, s);
    } else {
      const float* b = l == 0 ? R32 : (const float*)W.lb[l];
      if (L.vstore == VAL_BF16)
        m_pre(H, vec, K, L, view<__nv_bfloat16>(L.A, L.ah16), b, r, s);
      else
        m_pre(H, vec, K, L, view<float>(L.A, L.ah32), b, r, s);
    }
    AMG_LAUNCH_CHECK();
    if (vec)
      k_m_restrict_v<T><<<grid_for(L.nc * (K / (16 / (int)sizeof(T))), 256, H->num_sms, 8), 256,
                          0, s>>>(L.nc, L.stride, K, L.members, r, (T*)W.lb[l + 1]);
    else
      k_m_restrict<T><<<grid_for(L.nc * K, 256, H->num_sms, 8), 256, 0, s>>>(
          L.nc, L.stride, K, L.members, r, (T*)W.lb[l + 1]);
    AMG_LAUNCH_CHECK();
  }
  AMG_TRY(coarse((const T*)W.lb[nl - 1], (T*)W.lx[nl - 1]));
  for (int l = nl - 2; l >= 0; --l) {
    const Level& L = H->L[l];
    const T* xc = (const T*)W.lx[l + 1];
    if constexpr (sizeof(T) == 8) {
      const SellView<double> v = view<double>(L.AP, L.AP.v64);
      if (l == 0 && dots)
        m_post<true>(H, W, vec, K, L, v, R0, xc, Z0, Q, epi, s);
      else if (l == 0)
        m_post<false>(H, W, vec, K, L, v, R0, xc, Z0, Q, epi, s);
      else
        m_post<false>(H, W, vec, K, L, v, (const double*)W.lb[l], xc, (double*)W.lx[l], Q, epi,
                      s);
    } else {
      if (l == 0) {
        const SellView<float> v = view<float>(L.AP, L.AP.v32);
        if (dots)
          m_post<true>(H, W, vec, K, L, v, R0, xc, Z0, Q, epi, s);
        else
          m_post<false>(H, W, vec, K, L, v, R0, xc, Z0, Q, epi, s);
      } else if (L.vstore == VAL_BF16) {
        m_post<false>(H, W, vec, K, L, view<__nv_bfloat16>(L.AP, L.AP.v16),
                      (const float*)W.lb[l], xc, (float*)W.lx[l], Q, epi, s);
      } else {
        m_post<false>(H, W, vec, K, L, view<float>(L.AP, L.AP.v32), (const float*)W.lb[l], xc,
                      (float*)W.lx[l], Q, epi, s);
      }
    }
    AMG_LAUNCH_CHECK();
  }
  return AMG_OK;
}

static int m_vcycle_any(const amg_handle* H, const MultiWs& W, const double* R0, double* Z0,
                        bool dots, const double* Q, int beta_form, bool first, cudaStream_t s,
                        const float* R32 = nullptr) {
  if (H->opt.precision == AMG_PREC_F32)
    return m_vcycle<float>(H, W, R0, Z0, dots, Q, beta_form, first, s, R32);
  return m_vcycle<double>(H, W, R0, Z0, dots, Q, beta_form, first, s, nullptr);
}

// Workspace for K right-hand sides, kept in the handle (reallocated if K grows).
static int multi_ws(amg_handle* H, int K, MultiWs** out) {
  MultiWs* W = (MultiWs*)H->multi;
  if (W && W->K >= K) {
    W->K = K;
    *out = W;
    return AMG_OK;
  }
  if (W) {  // grow: drop the old buffers
    Arena& ar = H->arena;
    for (void* p : {(void*)W->R, (void*)W->R32, (void*)W->Z, (void*)W->P, (void*)W->Q,
                    (void*)W->cy,
                    (void*)W->part, (void*)W->ticket, (void*)W->sc, (void*)W->nactive})
      ar.release(p);
    for (size_t l = 0; l < H->L.size(); ++l) {
      ar.release(W->lb[l]);
      ar.release(W->lx[l]);
      ar.release(W->lr[l]);
    }
    delete[] W->lb;
    delete[] W->lx;
    delete[] W->lr;
    if (W->sc_host) cudaFreeHost(W->sc_host);
    delete W;
    H->multi = nullptr;
  }
  W = new MultiWs();
  H->multi = W;
  W->K = K;
  Arena& ar = H->arena;
  const int64_t n = H->L[0].n;
  const size_t vb = H->opt.precision == AMG_PREC_F32 ? 4 : 8;
  AMG_TRY(ar.alloc_n(&W->R, n * K));
  if (H->opt.precision == AMG_PREC_F32 && H->L.size() > 1) AMG_TRY(ar.alloc_n(&W->R32, n * K));
  AMG_TRY(ar.alloc_n(&W->Z, n * K));
  AMG_TRY(ar.alloc_n(&W->P, n * K));
  AMG_TRY(ar.alloc_n(&W->Q, n * K));
  AMG_TRY(ar.alloc_n(&W->cy, H->nco * K));
  AMG_TRY(ar.alloc_n(&W->part, (int64_t)2 * H->red.max_blocks * K));
  AMG_TRY(ar.alloc_n(&W->ticket, 1));
  AMG_TRY(ar.alloc_n(&W->sc, K));
  AMG_TRY(ar.alloc_n(&W->nactive, 1));
  AMG_CUDA_TRY(cudaMemset(W->ticket, 0, sizeof(unsigned)));
  AMG_CUDA_TRY(cudaMallocHost((void**)&W->sc_host, sizeof(Scal) * K));
  const size_t nl = H->L.size();
  W->lb = new void*[nl]();
  W->lx = new void*[nl]();
  W->lr = new void*[nl]();
  for (size_t l = 0; l < nl; ++l) {
    const size_t bytes = vb * (size_t)H->L[l].n * K;
    AMG_TRY(ar.alloc(&W->lb[l], bytes));
    AMG_TRY(ar.alloc(&W->lx[l], bytes));
    AMG_TRY(ar.alloc(&W->lr[l], bytes));
  }
  *out = W;
  return AMG_OK;
}

void multi_free(amg_handle* H) {
  MultiWs* W = (MultiWs*)H->multi;
  if (!W) return;
  delete[] W->lb;
  delete[] W->lx;
  delete[] W->lr;
  if (W->sc_host) cudaFreeHost(W->sc_host);
  delete W;
  H->multi = nullptr;
}

int vcycle_multi(amg_handle* H, int K, const double* R, double* Z, cudaStream_t s) {
  MultiWs* W = nullptr;
  AMG_TRY(multi_ws(H, K, &W));
  if (W->R32) {  // FP32 V-cycle: R rounded to FP32 once
    const int64_t m = H->L[0].n * K;
    const bool vec = (((uintptr_t)R | (uintptr_t)W->R32) & 15u) == 0;
    k_m_to_f32<<<grid_for((m + 3) / 4, 256, H->num_sms, 8), 256, 0, s>>>(m, R, W->R32, vec);
    AMG_LAUNCH_CHECK();
  }
  return m_vcycle_any(H, *W, R, Z, false, nullptr, PCG_BETA_FR, true, s, W->R32);
}

int pcg_multi_run(amg_handle* H, int K, const double* B, double* X, const pcg_options* o,
                  pcg_stats* st, cudaStream_t s) {
  MultiWs* W = nullptr;
  AMG_TRY(multi_ws(H, K, &W));
  const int64_t n = H->L[0].n;
  const Level& L0 = H->L[0];
  if (L0.A.row0) return AMG_ERR_UNSUPPORTED;  // batched handles: use pcg_solve_batch
  int beta_form = o->beta_form;
  if (beta_form == PCG_BETA_AUTO)
    beta_form = H->opt.precision == AMG_PREC_F32 ? PCG_BETA_FLEXIBLE : PCG_BETA_FR;
  const int maxb = H->red.max_blocks;
  const SellView<double> A = view<double>(L0.A, L0.A.v64);
  const int C = L0.A.C;
  const int g = mgrid(H, n), gmv = mgrid_mv(H, n);
  AMG_CUDA_TRY(cudaEventRecord(H->ev0, s));
  AMG_CUDA_TRY(cudaMemsetAsync(W->nactive, 0, sizeof(int), s));
  MultiInitEpi ie{W->sc, o->tol, o->maxit, W->nactive, 0};
  AMG_DISPATCH_KPL(K, (k_m_residual<KPL><<<gmv, MROWS_BLOCK, 0, s>>>(
                          A, C, K, B, X, W->R, W->part, maxb, W->ticket, ie, W->R32)));
  AMG_LAUNCH_CHECK();
  int act = 0;
  auto read_act = [&]() -> int {
    AMG_CUDA_TRY(cudaMemcpyAsync(&act, W->nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    return AMG_OK;
  };
  AMG_TRY(read_act());
  MultiPqEpi pe{W->sc};
  MultiRrEpi re{W->sc, o->tol, o->maxit, W->nactive};
  int k = 0;
  if (act > 0) {
    AMG_TRY(m_vcycle_any(H, *W, W->R, W->Z, true, W->Q, beta_form, true, s, W->R32));
    AMG_CUDA_TRY(cudaMemcpyAsync(W->P, W->Z, sizeof(double) * n * K, cudaMemcpyDeviceToDevice, s));
    for (;;) {
      if (K % 2 == 0)  // two doubles a lane (the workspace is 16-byte aligned)
        k_m_spmm_dot_v<<<gmv, MROWS_BLOCK, 0, s>>>(A, C, K, W->P, W->Q, W->part, maxb,
                                                  W->ticket, pe);
      else
        AMG_DISPATCH_KPL(K, (k_m_spmm_dot<KPL><<<gmv, MROWS_BLOCK, 0, s>>>(
                                A, C, K, W->P, W->Q, W->part, maxb, W->ticket, pe)));
      AMG_LAUNCH_CHECK();
      AMG_CUDA_TRY(cudaMemsetAsync(W->nactive, 0, sizeof(int), s));
      AMG_DISPATCH_KPL(K, (k_m_update<KPL><<<g, MROWS_BLOCK, 0, s>>>(n, K, X, W->R, W->P, W->Q,
                                                                    W->sc, W->part, maxb,
                                                                    W->ticket, re, W->R32)));
      AMG_LAUNCH_CHECK();
      ++k;
      AMG_TRY(read_act());
      if (act == 0 || k >= o->maxit) break;
      AMG_TRY(m_vcycle_any(H, *W, W->R, W->Z, true, W->Q, beta_form, false, s, W->R32));
      AMG_DISPATCH_KPL(K, (k_m_p_update<KPL><<<g, MROWS_BLOCK, 0, s>>>(n, K, W->P, W->Z, W->sc)));
      AMG_LAUNCH_CHECK();
    }
  }
  AMG_CUDA_TRY(cudaEventRecord(H->ev1, s));
  MultiInitEpi te{W->sc, o->tol, o->maxit, W->nactive, 1};
  AMG_DISPATCH_KPL(K, (k_m_residual<KPL><<<gmv, MROWS_BLOCK, 0, s>>>(
                          A, C, K, B, X, W->Z, W->part, maxb, W->ticket, te, nullptr)));
  AMG_LAUNCH_CHECK();
  AMG_CUDA_TRY(cudaMemcpyAsync(W->sc_host, W->sc, sizeof(Scal) * K, cudaMemcpyDeviceToHost, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  float ms = 0.f;
  AMG_CUDA_TRY(cudaEventElapsedTime(&ms, H->ev0, H->ev1));
  int worst = AMG_OK;
  for (int c = 0; c < K; ++c) {
    const Scal& S = W->sc_host[c];
    const double bn = S.bb > 0.0 ? sqrt(S.bb) : 1.0;
    if (st) {
      st[c].iterations = S.iters;
      st[c].status = S.status;
      st[c].rel_residual = sqrt(S.rr) / bn;
      st[c].true_rel_residual = sqrt(S.tr) / bn;
      st[c].solve_ms = ms;
    }
    if (S.status < 0 && (worst >= 0 || S.status < worst)) worst = S.status;
    if (S.status == AMG_NOT_CONVERGED && worst == AMG_OK) worst = AMG_NOT_CONVERGED;
  }
  return worst;
}

}  // namespace amg
