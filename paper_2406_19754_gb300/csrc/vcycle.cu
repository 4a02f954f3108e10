// The V(1,1) cycle of Eq. (amg) with zero initial guess on every level:
//
//   x = S b;  r = b - A x;  b_c = P^T r;  x_c = V(b_c);  x += P x_c;
//   x += S (b - A x),       S = diag(s), s_i = omega_i / (l1 row sum)_i,
//
// where P is the 0/1 aggregate map, and the coarsest level is solved by its
// dense Cholesky factor.  Each level streams two operators built at setup,
//   Ah = A S   (a_ij s_j)  and  AP = A P  (row i, column J: sum of a_ij over
//   agg(j) = J),
// so that every matrix entry needs exactly one gathered vector element:
//   k_pre      r = b - Ah b                 (= b - A (S b): pre-smooth + residual)
//   k_restrict b_c[I] = sum of r_i over the members of I, ascending
//   k_post     z = S b + P x_c + S (r - AP x_c)
// The last line is y + S (b - A y) for y = S b + P x_c, because
// b - A y = (b - A S b) - A P x_c.  The level-0 k_post can also reduce (r, z)
// and (z, q) for the PCG step.
#include <algorithm>

#include "ring.cuh"
#include "smooth.cuh"

namespace amg {

// ------------------------------------------------------------------ kernels

template <int TPR, typename V, typename T, typename BT>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_pre(SellView<V> Ah, const BT* __restrict__ b, T* __restrict__ r) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < Ah.ngroups;
       sl += nw)
    if (Ah.live(sl)) pre_slice<TPR, LdRO>(Ah, b, r, sl, ln);
}

template <typename T>
__global__ void k_restrict(int64_t nc, int stride, const int32_t* __restrict__ members,
                           const T* __restrict__ r, T* __restrict__ bc) {
  for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < nc;
       I += (int64_t)gridDim.x * blockDim.x)
    bc[I] = restrict_sum<LdRO>(members + I * stride, stride, r);
}

// Epilogue of the level-0 post-smoother when it feeds PCG: t[0] = (r, z),
// t[1] = (z, q).  beta = (r+, z+)/(r, z) or, flexible, -(z+, q)/(p, q).
struct VcycleDotEpi {
  PcgScalars* sc;
  template <int NV>
  __device__ void operator()(double (&t)[NV]) const {
    const double rz = t[0];
    const double zq = NV > 1 ? t[NV > 1 ? 1 : 0] : 0.0;
    const double beta = sc->beta_form == PCG_BETA_FLEXIBLE ? -zq / sc->pq : rz / sc->rz;
    sc->beta = beta;
    sc->zq = zq;
    sc->rz = rz;
    if (!isfinite(rz) && sc->status == 0) sc->status = AMG_ERR_NAN;
  }
};

// MS: the level smooths more than once per side (xp and e are used); the
// one-sweep instantiations do not carry them, which keeps their registers
// within the occupancy bound.  NDOT > 0 (level 0 of PCG): the kernel also
// forms (r, z) and, for NDOT = 2, (z, q), as grid-wide sums with no
// warp-collective operation inside the streaming loop (a per-slice warp
// reduction there cost 10% on 256^3 Poisson).  Batched systems use
// k_post_chunks below.
template <int TPR, typename V, typename T, typename BT, typename XT, int NDOT, bool MS>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_post(SellView<V> AP, const BT* __restrict__ b, const T* __restrict__ s,
           const T* __restrict__ r, const int32_t* __restrict__ agg, const T* __restrict__ xc,
           XT* __restrict__ x, const double* __restrict__ q, Reduce red, PcgScalars* sc,
           const T* __restrict__ xp, T* __restrict__ e) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  constexpr int ND = NDOT > 0 ? NDOT : 1;
  // the running sums sit in shared memory (one slot per thread, the same
  // additions in the same order as registers would do): the streaming loop
  // already fills the 32-register budget of full occupancy
  __shared__ double dacc[ND][NDOT > 0 ? SELL_BLOCK : 1];
  if constexpr (NDOT > 0) {
#pragma unroll
    for (int k = 0; k < NDOT; ++k) dacc[k][threadIdx.x] = 0.0;
  }
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < AP.ngroups;
       sl += nw) {
    if (!AP.live(sl)) continue;  // warp-uniform
    XT zi;
    const int64_t i = post_slice<TPR, LdRO>(AP, b, s, r, agg, xc, x, sl, ln, zi,
                                            MS ? xp : nullptr, MS ? e : nullptr);
    if constexpr (NDOT > 0) {
      if (i >= 0) {
        dacc[0][threadIdx.x] += (double)b[i] * (double)zi;
        if (NDOT > 1) dacc[NDOT > 1 ? 1 : 0][threadIdx.x] += (double)zi * q[i];
      }
    }
  }
  if constexpr (NDOT > 0) {
    double d[ND];
#pragma unroll
    for (int k = 0; k < NDOT; ++k) d[k] = dacc[k][threadIdx.x];
    grid_reduce<NDOT>(d, red, VcycleDotEpi{sc});
  }
}

// The level-0 post-smoother of batched systems with (r, z) (and (z, q)) per
// chunk of BATCH_CHUNK slices of one system: a warp walks whole chunks,
// keeps the sums per thread over the chunk's slices and reduces once at its
// end into part[2 c], part[2 c + 1] (no warp reduction in the slice loop).
template <int TPR, typename V, typename T, typename BT, typename XT, int NDOT>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_post_chunks(SellView<V> AP, int64_t nchunks, const int64_t* __restrict__ chunk_off,
                  const BT* __restrict__ b, const T* __restrict__ s, const T* __restrict__ r,
                  const int32_t* __restrict__ agg, const T* __restrict__ xc,
                  XT* __restrict__ x, const double* __restrict__ q, double* __restrict__ part) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks;
       c += nw) {
    const int64_t s0 = chunk_off[c], s1 = chunk_off[c + 1];
    if (!AP.live(s0)) continue;  // warp-uniform: one system per chunk
    double d0 = 0.0, d1 = 0.0;
    for (int64_t sl = s0; sl < s1; ++sl) {
      XT zi;
      const int64_t i = post_slice<TPR, LdRO>(AP, b, s, r, agg, xc, x, sl, ln, zi);
      if (i >= 0) {
        d0 += (double)b[i] * (double)zi;
        if (NDOT > 1) d1 += (double)zi * q[i];
      }
    }
    d0 = warp_sum(d0);
    if (NDOT > 1) d1 = warp_sum(d1);
    if ((threadIdx.x & 31) == 0) {
      part[2 * c] = d0;
      if (NDOT > 1) part[2 * c + 1] = d1;
    }
  }
}

// k_pre and k_post (one sweep, one system, one thread per row, FP64 or FP32
// operator values) on the shared-memory ring of ring.cuh: the same row
// arithmetic in the same order, so the same bits as the per-lane-load
// kernels; the dot products of the level-0 post-smoother are summed per
// thread over the warp's slices, then per block and over blocks, as there
// (with this launch's grid).  k_pre loads its row's b before waiting for the
// slice; k_post's row operands s, r, b, agg (and q for the second dot
// product) come with the slice (per-row vectors of the ring).
template <typename V, typename T, typename BT>
__global__ void __launch_bounds__(RING_THREADS, 4)
    k_pre_ring(SellView<V> Ah, const BT* __restrict__ b, T* __restrict__ r, RingGeom g,
               RingRows rows, int* fail) {
  extern __shared__ unsigned char ring_smem[];
  if (*(volatile int*)fail) return;
  RingWarp<V> ring(Ah, g, rows, ring_smem);
  ring.start();
  for (int64_t sl = ring.first; sl < Ah.nslices; sl += ring.nwt) {
    const int64_t i = sl * 32 + ring.lane;
    const bool has = i < Ah.n;
    const T bi = has ? to_f(__ldg(b + i), T(0)) : T(0);  // overlaps the wait
    if (!ring.wait()) {
      if (ring.lane == 0) ring_fail(fail, nullptr);
      ring.drain();
      return;
    }
    // pre_slice's arithmetic: from b_i down by negated FMAs
    const T acc = ring_row_sum<T, true>(
        ring, ring.width(), [&](int j) { return to_f(__ldg(b + j), T(0)); }, bi);
    if (has) r[i] = acc;
    ring.release();
  }
}

template <typename V, typename T, typename BT, typename XT, int NDOT>
__global__ void __launch_bounds__(RING_THREADS, 4)
    k_post_ring(SellView<V> AP, const BT* __restrict__ b, const T* __restrict__ s,
                const T* __restrict__ r, const int32_t* __restrict__ agg,
                const T* __restrict__ xc, XT* __restrict__ x, const double* __restrict__ q,
                Reduce red, PcgScalars* sc, RingGeom g, RingRows rows, int* fail) {
  extern __shared__ unsigned char ring_smem[];
  if (*(volatile int*)fail) return;  // the host resets the reduction ticket
  constexpr int ND = NDOT > 0 ? NDOT : 1;
  double d[ND];
#pragma unroll
  for (int k = 0; k < ND; ++k) d[k] = 0.0;
  RingWarp<V> ring(AP, g, rows, ring_smem);
  ring.start();
  for (int64_t sl = ring.first; sl < AP.nslices; sl += ring.nwt) {
    if (!ring.wait()) {
      if (ring.lane == 0) ring_fail(fail, NDOT > 0 ? &sc->status : nullptr);
      ring.drain();
      break;
    }
    const bool f = ring.full(sl);
    const int64_t i = sl * 32 + ring.lane;
    const bool has = i < AP.n;
    T si = T(0), ri = T(0);
    BT bi = BT(0);
    int32_t ai = 0;
    double qi = 0.0;
    if (has) {  // the row's operands, which came with the slice
      si = ring.template row<T>(0, f, i);
      ri = ring.template row<T>(1, f, i);
      bi = ring.template row<BT>(2, f, i);
      ai = ring.template row<int32_t>(3, f, i);
      if constexpr (NDOT > 1) qi = ring.template row<double>(4, f, i);
    }
    // x_c of the row's own aggregate: gathered with the row's entries
    const T xci = has ? __ldg(xc + ai) : T(0);
    // post_slice's arithmetic (one sweep): from b_i + r_i down, then one FMA
    const T init = has ? to_f(bi, T(0)) + ri : T(0);
    const T acc =
        ring_row_sum<T, true>(ring, ring.width(), [&](int J) { return __ldg(xc + J); }, init);
    if (has) {
      const XT zi = to_f(fma(si, acc, xci), XT(0));
      x[i] = zi;
      if constexpr (NDOT > 0) d[0] += (double)bi * (double)zi;
      if constexpr (NDOT > 1) d[NDOT > 1 ? 1 : 0] += (double)zi * qi;
    }
    ring.release();
  }
  if constexpr (NDOT > 0) grid_reduce<NDOT>(d, red, VcycleDotEpi{sc});
}

// Post-smoother of a level with a smoothed prolongator P (Sec. 2.3; A P in
// AQ, P with the same slices): z = y + S (r - (A P) x_c), y = x_pre + P x_c,
// x_pre the pre-smoothed x (xp, or S b after one sweep); e, if set, receives
// r - (A P) x_c for further sweeps.  V: stored values, T: V-cycle vectors,
// BT / XT: this level's b and output (FP64 on level 0).
template <int TPR, typename V, typename T, typename BT, typename XT>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_post_sm(SellView<V> AQ, SellView<V> P, const BT* __restrict__ b,
              const T* __restrict__ s, const T* __restrict__ r, const T* __restrict__ xc,
              const T* __restrict__ xp, XT* __restrict__ x, T* __restrict__ e) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < AQ.ngroups;
       sl += nw) {
    const T aq = sell_row<TPR, T>(AQ, sl, ln, [&](int J) { return __ldg(xc + J); });
    const T px = sell_row<TPR, T>(P, sl, ln, [&](int J) { return __ldg(xc + J); });
    const int64_t i = lane_row(AQ, sl, ln);
    if (i >= 0) {
      const T si = s[i];
      const T yi = (xp ? xp[i] : si * to_f(b[i], T(0))) + px;
      const T ei = r[i] - aq;
      x[i] = to_f(fma(si, ei, yi), XT(0));
      if (e) e[i] = ei;
    }
  }
}

// b_c = R r for a smoothed level (R = P^T, own slices); V-cycle vector types.
template <int TPR, typename V, typename T>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_restrict_sm(SellView<V> R, const T* __restrict__ r, T* __restrict__ bc) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < R.ngroups;
       sl += nw) {
    const T acc = sell_row<TPR, T>(R, sl, ln, [&](int j) { return __ldg(r + j); });
    const int64_t I = lane_row(R, sl, ln);
    if (I >= 0) bc[I] = acc;
  }
}

// Pre-smoothing sweeps 2..nu on the residual recurrence: x += S r (x = S b
// before the first of them), r_out = r - (A S) r.
template <int TPR, typename V, typename T, typename BT>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_sweep_pre(SellView<V> Ah, const T* __restrict__ s, const BT* __restrict__ b,
                const T* __restrict__ r, T* __restrict__ r_out, T* __restrict__ x, int first) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < Ah.ngroups;
       sl += nw) {
    if (!Ah.live(sl)) continue;
    T ri = T(0), rn = T(0);
    int64_t i;
    sweep_slice<TPR, LdRO>(Ah, s, r, r_out, sl, ln, ri, rn, i);
    if (i >= 0) {
      const T si = s[i];
      const T xi = first ? si * to_f(b[i], T(0)) : x[i];
      x[i] = sweep_pre_x(xi, si, ri);
    }
  }
}

// Post-smoothing sweeps 2..nu: r_out = r - (A S) r (the residual of y after
// its last update), then y += S r_out.
template <int TPR, typename V, typename T, typename YT>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_sweep_post(SellView<V> Ah, const T* __restrict__ s, const T* __restrict__ r,
                 T* __restrict__ r_out, YT* __restrict__ y) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < Ah.ngroups;
       sl += nw) {
    if (!Ah.live(sl)) continue;
    T ri = T(0), rn = T(0);
    int64_t i;
    sweep_slice<TPR, LdRO>(Ah, s, r, r_out, sl, ln, ri, rn, i);
    if (i >= 0) y[i] = sweep_post_y(y[i], s[i], rn);
  }
}

static __global__ void k_vec_to_f32(int64_t n, const double* __restrict__ v,
                                    float* __restrict__ w) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = (float)v[i];
}

// Groups of four elements, as the blocked kernels convert them: an input out
// of the bit path's range sends its whole group to the hardware conversion.
static __global__ void k_debug_convert(int64_t n, const double* __restrict__ in64,
                                       float* __restrict__ out32, const float* __restrict__ in32,
                                       double* __restrict__ out64) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; 4 * t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = 4 * t;
    const int m = (int)(n - i < 4 ? n - i : 4);
    if (in64) {
      double a[4];
      float b[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = k < m ? in64[i + k] : 0.0;
      cvt_n(a, b);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < m) out32[i + k] = b[k];
    }
    if (in32) {
      float a[4];
      double b[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = k < m ? in32[i + k] : 0.0f;
      cvt_n(a, b);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k < m) out64[i + k] = b[k];
    }
  }
}

// Dots for the single-level case (the whole preconditioner is the coarse solve).
template <int NDOT>
__global__ void k_dots_rz(int64_t n, const double* r, const double* z, const double* q, Reduce red,
                          PcgScalars* sc) {
  double d[NDOT];
#pragma unroll
  for (int k = 0; k < NDOT; ++k) d[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    d[0] += r[i] * z[i];
    if (NDOT > 1) d[NDOT > 1 ? 1 : 0] += z[i] * q[i];
  }
  grid_reduce<NDOT>(d, red, VcycleDotEpi{sc});
}

// Per-chunk (r, z) and (z, q) partials over the level-0 chunks of batched
// systems (see Batch), for V-cycles whose level-0 post-smoother does not
// form them.
template <int NDOT>
__global__ void k_chunk_dots(SellView<double> A, int64_t nchunks,
                             const int64_t* __restrict__ chunk_off, const double* r,
                             const double* z, const double* q, double* part) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks;
       c += nw) {
    // the chunk's rows are contiguous (system-aligned slices)
    const int64_t b0 = A.rbeg(chunk_off[c], 32), b1 = A.rend(chunk_off[c + 1] - 1, 32);
    double d0 = 0.0, d1 = 0.0;
    for (int64_t i = b0 + lane; i < b1; i += 32) {
      d0 += r[i] * z[i];
      if (NDOT > 1) d1 += z[i] * q[i];
    }
    d0 = warp_sum(d0);
    if (NDOT > 1) d1 = warp_sum(d1);
    if (lane == 0) {  // two slots per chunk, as every batched reduction uses
      part[c * 2] = d0;
      if (NDOT > 1) part[c * 2 + 1] = d1;
    }
  }
}

static int slice_dots(const amg_handle* H, const double* r, const double* z, const double* q,
                      int dots, double* part, cudaStream_t s) {
  // rbeg/rend with C = 32 are exact for system-aligned slices (row0 set)
  const Level& L = H->L[0];
  const Batch& B = H->batch;
  if (!L.A.row0 || !B.chunk_off) return AMG_ERR_ARG;
  const SellView<double> v = view<double>(L.A, L.A.v64);
  const int grid = sell_grid(B.nchunks, H->num_sms);
  if (dots == 1)
    k_chunk_dots<1><<<grid, SELL_BLOCK, 0, s>>>(v, B.nchunks, B.chunk_off, r, z, q, part);
  else
    k_chunk_dots<2><<<grid, SELL_BLOCK, 0, s>>>(v, B.nchunks, B.chunk_off, r, z, q, part);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// Coarsest level: x = L^-T (L^-1 b), one CUDA block per diagonal block.
template <typename BT, typename XT>
__global__ void k_coarse(const int64_t* __restrict__ brow, const int64_t* __restrict__ bmat,
                         const double* __restrict__ Linv_all,
                         const double* __restrict__ LinvT_all, const BT* __restrict__ b_all,
                         XT* __restrict__ x_all, const int* __restrict__ act) {
  extern __shared__ double csh[];
  if (act && !act[blockIdx.x]) return;  // block = system of a batch; stopped
  coarse_block_solve<LdRO>(blockIdx.x, brow, bmat, Linv_all, LinvT_all, b_all, x_all, csh);
}

// Large coarsest blocks: y = L^-1 b, then x = L^-T y, one warp per row over
// the whole GPU.
template <typename BT>
__global__ void k_coarse_y(int64_t nco, int nblk, const int64_t* __restrict__ brow,
                           const int64_t* __restrict__ bmat, const double* __restrict__ Linv_all,
                           const BT* __restrict__ b, double* __restrict__ y) {
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nco; g += nw)
    coarse_y_row<LdRO>(g, nblk, brow, bmat, Linv_all, b, y);
}

template <typename XT>
__global__ void k_coarse_x(int64_t nco, int nblk, const int64_t* __restrict__ brow,
                           const int64_t* __restrict__ bmat,
                           const double* __restrict__ LinvT_all, const double* __restrict__ y,
                           XT* __restrict__ x) {
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < nco; g += nw)
    coarse_x_row<LdRO>(g, nblk, brow, bmat, LinvT_all, y, x);
}

// Coarsest solve by PCG with the l1-Jacobi preconditioner in one CUDA block
// (coarse_pcg_cta).  w null: the five work vectors live in dynamic shared
// memory (latency-bound iterations; the same arithmetic either way).
template <int TPR, typename BT, typename XT>
__global__ void __launch_bounds__(1024, 1)
    k_coarse_pcg(SellView<double> A, const double* __restrict__ sinv, const BT* __restrict__ b,
                 XT* __restrict__ xo, double* w, int maxit, double tol) {
  extern __shared__ double wsh[];
  coarse_pcg_cta<TPR>(A, sinv, b, xo, w ? w : wsh, maxit, tol);
}

// Largest PCG coarsest level whose work vectors go to shared memory (within
// the default 48 KB of dynamic shared memory, so no attribute call is needed
// while a graph is being captured).
constexpr int64_t COARSE_PCG_SMEM_ROWS = 1152;  // 5 x 1152 doubles = 45 KB, plus the static sums

// ------------------------------------------------------------------ driver

template <typename BT, typename XT>
static int coarse_solve(const amg_handle* H, const BT* b, XT* x, cudaStream_t s,
                        const int* act = nullptr) {
  if (H->opt.coarse_solver == 1) {  // PCG with l1-Jacobi (non-batched handles only)
    const Level& Lc = H->L.back();
    const SellView<double> v = view<double>(Lc.A, Lc.A.v64);
    const bool sh = Lc.n <= COARSE_PCG_SMEM_ROWS;
    const size_t smem = sh ? sizeof(double) * 5 * (size_t)Lc.n : 0;
    double* w = sh ? nullptr : H->cpcg;
    AMG_DISPATCH_TPR(sell_code(Lc.A), (k_coarse_pcg<TPR, BT, XT><<<1, 1024, smem, s>>>(
                                          v, Lc.s64, b, x, w, H->opt.coarse_maxit,
                                          H->opt.coarse_tol)));
    AMG_LAUNCH_CHECK();
    return AMG_OK;
  }
  int64_t m = 0;  // largest block
  for (int k = 0; k < H->nblk; ++k) m = std::max(m, H->cblk_row[k + 1] - H->cblk_row[k]);
  if (m <= COARSE_SMALL) {  // one CUDA block per diagonal block; 2m doubles <= 16 KB
    const size_t sm = sizeof(double) * 2 * (size_t)m;
    k_coarse<BT, XT><<<H->nblk, 1024, sm, s>>>(H->d_brow, H->d_bmat, H->Linv, H->LinvT, b, x,
                                               act);
    AMG_LAUNCH_CHECK();
    return AMG_OK;
  }
  const int grid = grid_for(H->nco * 32, 256, H->num_sms, 8);
  k_coarse_y<BT><<<grid, 256, 0, s>>>(H->nco, H->nblk, H->d_brow, H->d_bmat, H->Linv, b,
                                      H->coarse_y);
  AMG_LAUNCH_CHECK();
  k_coarse_x<XT><<<grid, 256, 0, s>>>(H->nco, H->nblk, H->d_brow, H->d_bmat, H->LinvT,
                                      H->coarse_y, x);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// act: per-system active flags of a batched PCG (slices of stopped systems
// are skipped), or null.
template <typename V, typename T, typename BT>
static int launch_pre(const amg_handle* H, const Level& L, const V* ah, const BT* b, T* r,
                      cudaStream_t s, const int* act = nullptr) {
  const int grid = sell_grid(sell_groups(L.A), H->num_sms);
  SellView<V> v = view<V>(L.A, ah);
  v.act = act;
  // FP64 and FP32 operators (BF16 values keep the per-lane kernels)
  if constexpr (sizeof(V) >= 4) {
    if (!act && H->opt.stream_ring) {
      RingGeom g = ring_plan(L.A, (int)sizeof(V), ring_stages(H), RingRows());
      if (g.D) {
        AMG_TRY(ring_prepare((const void*)k_pre_ring<V, T, BT>, g, L.A.nslices, H->num_sms));
        k_pre_ring<V, T, BT><<<g.grid, RING_THREADS, g.smem, s>>>(v, b, r, g, RingRows(),
                                                                 H->wait_fail);
        AMG_LAUNCH_CHECK();
        return AMG_OK;
      }
    }
  }
  AMG_DISPATCH_TPR(sell_code(L.A),
                   (k_pre<TPR, V, T, BT><<<grid, SELL_BLOCK, 0, s>>>(v, b, r)));
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// Post-smoother operands of a level with several sweeps: the final
// pre-smoothing residual, the pre-smoothed x, and where the residual of
// y = xp + P x_c goes (null for one sweep: r is L.r and xp is S b).
template <typename T>
struct PostIn {
  const T* r = nullptr;
  const T* xp = nullptr;
  T* e = nullptr;
};

template <typename V, typename T, typename BT, typename XT, int NDOT>
static int launch_post(const amg_handle* H, const Level& L, const V* ap, const BT* b,
                       const T* xc, XT* x, const double* q, cudaStream_t s,
                       double* slice_part, const int* act, const PostIn<T>& in) {
  const int grid = sell_grid(sell_groups(L.AP), H->num_sms);
  SellView<V> v = view<V>(L.AP, ap);
  v.act = act;
  const T* sc = (const T*)(sizeof(T) == 8 ? (const void*)L.s64 : (const void*)L.s32);
  const T* r = in.r ? in.r : (const T*)L.r;
  if constexpr (NDOT == 0) {
    if (in.xp) {
      AMG_DISPATCH_TPR(sell_code(L.AP),
                       (k_post<TPR, V, T, BT, XT, 0, true><<<grid, SELL_BLOCK, 0, s>>>(
                           v, b, sc, r, L.agg, xc, x, q, H->red, H->sc, in.xp, in.e)));
      AMG_LAUNCH_CHECK();
      return AMG_OK;
    }
  }
  if (in.xp) return AMG_ERR_ARG;  // several sweeps: the dot products follow separately
  if constexpr (sizeof(V) >= 4) {  // FP64 and FP32 operators, as for k_pre
    if (!act && !slice_part && H->opt.stream_ring) {
      RingRows rows;  // indices 0..4 as read by k_post_ring
      rows.add(sc, (int)sizeof(T));
      rows.add(r, (int)sizeof(T));
      rows.add(b, (int)sizeof(BT));
      rows.add(L.agg, (int)sizeof(int32_t));
      if (NDOT > 1) rows.add(q, (int)sizeof(double));
      RingGeom g = ring_plan(L.AP, (int)sizeof(V), ring_stages(H), rows);
      if (g.D) {
        AMG_TRY(ring_prepare((const void*)k_post_ring<V, T, BT, XT, NDOT>, g, L.AP.nslices,
                             H->num_sms));
        k_post_ring<V, T, BT, XT, NDOT><<<g.grid, RING_THREADS, g.smem, s>>>(
            v, b, sc, r, L.agg, xc, x, q, H->red, H->sc, g, rows, H->wait_fail);
        AMG_LAUNCH_CHECK();
        return AMG_OK;
      }
    }
  }
  if constexpr (NDOT > 0) {
    if (slice_part) {  // batched systems: per-chunk partials
      const Batch& B = H->batch;
      if (!B.chunk_off) return AMG_ERR_ARG;
      const int cg = sell_grid(B.nchunks, H->num_sms);
      AMG_DISPATCH_TPR(sell_code(L.AP),
                       (k_post_chunks<TPR, V, T, BT, XT, NDOT><<<cg, SELL_BLOCK, 0, s>>>(
                           v, B.nchunks, B.chunk_off, b, sc, r, L.agg, xc, x, q, slice_part)));
      AMG_LAUNCH_CHECK();
      return AMG_OK;
    }
  }
  AMG_DISPATCH_TPR(sell_code(L.AP),
                   (k_post<TPR, V, T, BT, XT, NDOT, false><<<grid, SELL_BLOCK, 0, s>>>(
                       v, b, sc, r, L.agg, xc, x, q, H->red, H->sc, nullptr, nullptr)));
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// One further pre- (PRE) or post-smoothing sweep of level L on the residual
// recurrence (k_sweep_pre / k_sweep_post).
template <bool PRE, typename T, typename BT, typename YT>
static int launch_sweep(const amg_handle* H, const Level& L, const BT* b, const T* r, T* r_out,
                        YT* x, int first, cudaStream_t s, const int* act) {
  const int grid = sell_grid(sell_groups(L.A), H->num_sms);
  const T* sc = (const T*)(sizeof(T) == 8 ? (const void*)L.s64 : (const void*)L.s32);
  auto go = [&](auto vtag, const auto* ah) -> int {
    using V = decltype(vtag);
    SellView<V> v = view<V>(L.A, ah);
    v.act = act;
    if constexpr (PRE) {
      AMG_DISPATCH_TPR(sell_code(L.A), (k_sweep_pre<TPR, V, T, BT><<<grid, SELL_BLOCK, 0, s>>>(
                                            v, sc, b, r, r_out, (T*)x, first)));
    } else {
      AMG_DISPATCH_TPR(sell_code(L.A), (k_sweep_post<TPR, V, T, YT><<<grid, SELL_BLOCK, 0, s>>>(
                                            v, sc, r, r_out, x)));
    }
    AMG_LAUNCH_CHECK();
    return AMG_OK;
  };
  if constexpr (sizeof(T) == 8) {
    return go(double(0), L.ah64);
  } else {
    if (L.vstore == VAL_BF16) return go(__nv_bfloat16(), L.ah16);
    return go(float(0), L.ah32);
  }
}

// Values of a smoothed-level operator in the level's storage type.
template <typename V>
static const V* sm_vals(const Sell& M) {
  if constexpr (sizeof(V) == 8) return M.v64;
  else if constexpr (sizeof(V) == 4) return M.v32;
  else return M.v16;
}

template <typename T>
static int launch_restrict(const amg_handle* H, const Level& L, const T* r, T* bc,
                           cudaStream_t s) {
  if (H->opt.smooth_prolongator) {  // b_c = R r, R = P^T
    const int grid = sell_grid(sell_groups(L.R), H->num_sms);
    auto go = [&](auto vtag) -> int {
      using V = decltype(vtag);
      const SellView<V> v = view<V>(L.R, sm_vals<V>(L.R));
      AMG_DISPATCH_TPR(sell_code(L.R),
                       (k_restrict_sm<TPR, V, T><<<grid, SELL_BLOCK, 0, s>>>(v, r, bc)));
      AMG_LAUNCH_CHECK();
      return AMG_OK;
    };
    if constexpr (sizeof(T) == 8) return go(double(0));
    else return L.vstore == VAL_BF16 ? go(__nv_bfloat16()) : go(float(0));
  }
  k_restrict<T><<<grid_for(L.nc, 256, H->num_sms, 8), 256, 0, s>>>(L.nc, L.stride, L.members, r,
                                                                   bc);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

template <typename BT>
static int pre_f32(const amg_handle* H, const Level& L, const BT* b, float* r, cudaStream_t s,
                   const int* act = nullptr) {
  if (L.vstore == VAL_BF16)
    return launch_pre<__nv_bfloat16, float, BT>(H, L, L.ah16, b, r, s, act);
  return launch_pre<float, float, BT>(H, L, L.ah32, b, r, s, act);
}

// Post-smoother of a smoothed-prolongator level (k_post_sm; no dot products).
template <typename T, typename BT, typename XT>
static int launch_post_sm(const amg_handle* H, const Level& L, const BT* b, const T* xc, XT* x,
                          cudaStream_t s, const PostIn<T>& in) {
  const int grid = sell_grid(sell_groups(L.AP), H->num_sms);
  const T* sc = (const T*)(sizeof(T) == 8 ? (const void*)L.s64 : (const void*)L.s32);
  const T* r = in.r ? in.r : (const T*)L.r;
  if (sell_code(L.AP) != sell_code(L.P)) return AMG_ERR_UNSUPPORTED;
  auto go = [&](auto vtag) -> int {
    using V = decltype(vtag);
    const SellView<V> q = view<V>(L.AP, sm_vals<V>(L.AP));
    const SellView<V> p = view<V>(L.P, sm_vals<V>(L.P));
    AMG_DISPATCH_TPR(sell_code(L.AP), (k_post_sm<TPR, V, T, BT, XT><<<grid, SELL_BLOCK, 0, s>>>(
                                          q, p, b, sc, r, xc, in.xp, x, in.e)));
    AMG_LAUNCH_CHECK();
    return AMG_OK;
  };
  if constexpr (sizeof(T) == 8) return go(double(0));
  else return L.vstore == VAL_BF16 ? go(__nv_bfloat16()) : go(float(0));
}

template <typename T, typename BT, typename XT, int NDOT>
static int post_any(const amg_handle* H, const Level& L, const BT* b, const T* xc, XT* x,
                    const double* q, cudaStream_t s, double* slice_part = nullptr,
                    const int* act = nullptr, const PostIn<T>& in = PostIn<T>()) {
  if constexpr (NDOT == 0) {
    if (H->opt.smooth_prolongator) return launch_post_sm<T, BT, XT>(H, L, b, xc, x, s, in);
  }
  if constexpr (sizeof(T) == 8) {
    return launch_post<double, T, BT, XT, NDOT>(H, L, L.AP.v64, b, xc, x, q, s, slice_part,
                                                 act, in);
  } else {
    if (L.vstore == VAL_BF16)
      return launch_post<__nv_bfloat16, T, BT, XT, NDOT>(H, L, L.AP.v16, b, xc, x, q, s,
                                                          slice_part, act, in);
    return launch_post<float, T, BT, XT, NDOT>(H, L, L.AP.v32, b, xc, x, q, s, slice_part,
                                                act, in);
  }
}

// Optional per-kernel timing: an event pair around every launch plus the
// kernel's algorithmic bytes (each array counted once per pass).
struct Prof {
  cudaStream_t s;
  std::vector<cudaEvent_t> ev;
  std::vector<amg_kernel_time> rec;
  int begin(int level, int kind, double bytes) {
    cudaEvent_t a, b;
    AMG_CUDA_TRY(cudaEventCreate(&a));
    AMG_CUDA_TRY(cudaEventCreate(&b));
    ev.push_back(a);
    ev.push_back(b);
    amg_kernel_time k;
    k.level = level;
    k.kind = kind;
    k.bytes = bytes;
    k.ms = 0.0;
    rec.push_back(k);
    AMG_CUDA_TRY(cudaEventRecord(a, s));
    return AMG_OK;
  }
  int end() {
    AMG_CUDA_TRY(cudaEventRecord(ev.back(), s));
    return AMG_OK;
  }
  int finish() {
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t k = 0; k < rec.size(); ++k) {
      float ms = 0.f;
      AMG_CUDA_TRY(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
      rec[k].ms = ms;
    }
    return AMG_OK;
  }
  ~Prof() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

// Algorithmic bytes of each V-cycle kernel on one level: operator entries
// (value + column index) once, every vector once.  mb = bytes of an operator
// entry (value + 4-byte column, or + 2-byte offset and a share of the 4-byte
// base per C slots when the columns are compressed), vb = bytes of a V-cycle
// vector element, ib/ob = bytes of the level's input b / output z elements
// (FP64 on level 0).
static double bytes_pre(const Level& L, double mb, double vb, double ib) {
  return (double)L.nnz * mb + (double)L.n * (ib + vb);  // Ah, b, r
}
// With a smoothed prolongator the restriction streams R = P^T (12 bytes an
// entry) instead of the member lists, and the post-smoother streams P in
// place of the aggregate map.
static double bytes_restrict(const Level& L, double vb) {
  if (L.R.nslices) return (double)L.p_nnz * 12.0 + (double)L.n * vb + (double)L.nc * vb;
  return (double)L.n * (vb + 4.0) + (double)L.nc * vb;  // r, members, b_c
}
static double bytes_post(const Level& L, double mb, double vb, double ib, double ob) {
  if (L.P.nslices)  // A P, P, b, s, r, z, x_c
    return (double)(L.ap_nnz + L.p_nnz) * mb + (double)L.n * (ib + vb + vb + ob) +
           (double)L.nc * vb;
  // AP, b, s, r, agg, z, x_c
  return (double)L.ap_nnz * mb + (double)L.n * (ib + vb + vb + 4.0 + ob) + (double)L.nc * vb;
}

// Triangles of L^-1 and L^-T read by the coarse solve (lower/upper halves of
// every diagonal block).
static double coarse_factor_bytes(const amg_handle* H) {
  if (H->opt.coarse_solver != 0) return 12.0 * (double)H->L.back().nnz;  // PCG: A per pass
  double t = 0.0;
  for (int k = 0; k < H->nblk; ++k) {
    const double m = (double)(H->cblk_row[k + 1] - H->cblk_row[k]);
    t += m * (m + 1.0) * 8.0;  // two triangles of m(m+1)/2 doubles
  }
  return t;
}

#define PROF_BEGIN(lvl, kind, bytes) \
  if (prof) AMG_TRY(prof->begin((lvl), (kind), (bytes)))
#define PROF_END() \
  if (prof) AMG_TRY(prof->end())

template <typename T>
static int vcycle_levels(const amg_handle* H, const double* r0, double* z0, int dots,
                         const double* q, cudaStream_t s, Prof* prof, double* slice_part,
                         const float* r32 = nullptr) {
  const int nl = (int)H->L.size();
  const double vb = sizeof(T);
  // batched PCG (slice partials requested): skip the systems that stopped
  const int* act = slice_part ? H->batch.active : nullptr;
  auto entry = [&](const Level& L, const Sell& M) {
    const double idx = M.d16 ? 2.0 + 4.0 / M.C : 4.0;
    return idx + (L.vstore == VAL_F64 ? 8.0 : L.vstore == VAL_F32 ? 4.0 : 2.0);
  };
  auto mbytes = [&](const Level& L) { return entry(L, L.A); };
  auto pbytes = [&](const Level& L) { return entry(L, L.AP); };
  // (r, z) and (z, q) for PCG when they are not fused into the last kernel
  auto separate_dots = [&]() -> int {
    if (dots > 0 && slice_part) {
      AMG_TRY(slice_dots(H, r0, z0, q, dots, slice_part, s));
    } else if (dots > 0) {
      const int grid = grid_for(H->L[0].n, 256, H->num_sms, 8);
      if (dots == 1)
        k_dots_rz<1><<<grid, 256, 0, s>>>(H->L[0].n, r0, z0, q, H->red, H->sc);
      else
        k_dots_rz<2><<<grid, 256, 0, s>>>(H->L[0].n, r0, z0, q, H->red, H->sc);
      AMG_LAUNCH_CHECK();
    }
    return AMG_OK;
  };
  if (nl == 1) {
    const double m = (double)H->nco;
    PROF_BEGIN(0, 3, coarse_factor_bytes(H) + m * 16.0);
    AMG_TRY(coarse_solve<double, double>(H, r0, z0, s, act));
    PROF_END();
    return separate_dots();
  }
  // Levels with nu > 1 sweeps alternate two residual buffers: cur[l] says
  // which one holds the current residual.
  std::vector<int> cur(nl, 0);
  auto rbuf = [&](const Level& L, int k) { return (T*)(k == 0 ? L.r : L.r2); };
  auto sweep_bytes = [&](const Level& L) {  // A S, r in and out, s, x read and written
    return (double)L.nnz * mbytes(L) + (double)L.n * 5.0 * vb;
  };
  // Levels lt .. coarsest run in one persistent launch (tail.cu) when the
  // handle allows it; the others get one launch per step.
  const int lt = tail_start(H);
  const int ldown = lt >= 0 ? lt : nl - 1;
  // downward: pre-smooth + residual, restriction
  for (int l = 0; l < ldown; ++l) {
    const Level& L = H->L[l];
    T* r = (T*)L.r;
    PROF_BEGIN(l, 0, bytes_pre(L, mbytes(L), vb, l > 0 ? vb : r32 ? 4.0 : 8.0));
    if constexpr (sizeof(T) == 8) {
      const double* b = l == 0 ? r0 : (const double*)L.b;
      AMG_TRY((launch_pre<double, double, double>(H, L, L.ah64, b, r, s, act)));
    } else {
      if (l == 0)
        AMG_TRY(r32 ? pre_f32<float>(H, L, r32, r, s, act)
                    : pre_f32<double>(H, L, r0, r, s, act));
      else
        AMG_TRY(pre_f32<float>(H, L, (const float*)L.b, r, s, act));
    }
    PROF_END();
    for (int64_t k = 2; k <= L.nu; ++k) {  // further pre-smoothing sweeps
      const int c = cur[l];
      PROF_BEGIN(l, 5, sweep_bytes(L));
      if (l > 0)
        AMG_TRY((launch_sweep<true, T, T, T>(H, L, (const T*)L.b, rbuf(L, c), rbuf(L, 1 - c),
                                             (T*)L.xp, k == 2, s, act)));
      else if (sizeof(T) == 4 && r32)
        AMG_TRY((launch_sweep<true, T, float, T>(H, L, r32, rbuf(L, c), rbuf(L, 1 - c),
                                                 (T*)L.xp, k == 2, s, act)));
      else
        AMG_TRY((launch_sweep<true, T, double, T>(H, L, r0, rbuf(L, c), rbuf(L, 1 - c),
                                                  (T*)L.xp, k == 2, s, act)));
      PROF_END();
      cur[l] = 1 - c;
    }
    PROF_BEGIN(l, 1, bytes_restrict(L, vb));
    AMG_TRY(launch_restrict<T>(H, L, rbuf(L, cur[l]), (T*)H->L[l + 1].b, s));
    PROF_END();
  }
  const double mc = (double)H->nco;
  if (lt >= 0) {
    double bytes = coarse_factor_bytes(H) + mc * 2.0 * vb;
    for (int l = lt; l < nl - 1; ++l) {
      const Level& L = H->L[l];
      bytes += bytes_pre(L, mbytes(L), vb, vb) + bytes_restrict(L, vb) +
               bytes_post(L, pbytes(L), vb, vb, vb) + 2.0 * (double)(L.nu - 1) * sweep_bytes(L);
    }
    PROF_BEGIN(lt, 4, bytes);
    AMG_TRY(tail_launch<T>(H, lt, s, act));
    PROF_END();
  } else {
    PROF_BEGIN(nl - 1, 3, coarse_factor_bytes(H) + mc * 2.0 * vb);
    AMG_TRY((coarse_solve<T, T>(H, (const T*)H->L[nl - 1].b, (T*)H->L[nl - 1].x, s, act)));
    PROF_END();
  }
  // The post-smoother of a level with nu > 1 sweeps: the first sweep also
  // keeps the residual of y = xp + P x_c, the others step the recurrence.
  auto post_in = [&](const Level& L, int l) {
    PostIn<T> in;
    if (L.nu > 1) {
      in.r = rbuf(L, cur[l]);
      in.xp = (const T*)L.xp;
      in.e = rbuf(L, 1 - cur[l]);
      cur[l] = 1 - cur[l];
    }
    return in;
  };
  auto post_sweeps = [&](const Level& L, int l, auto* y) -> int {
    for (int64_t m = 2; m <= L.nu; ++m) {
      const int c = cur[l];
      PROF_BEGIN(l, 5, sweep_bytes(L));
      AMG_TRY((launch_sweep<false, T, T>(H, L, (const T*)nullptr, rbuf(L, c), rbuf(L, 1 - c), y,
                                         0, s, act)));
      PROF_END();
      cur[l] = 1 - c;
    }
    return AMG_OK;
  };
  // upward: prolongation + post-smooth
  for (int l = ldown - 1; l >= 1; --l) {
    const Level& L = H->L[l];
    PROF_BEGIN(l, 2, bytes_post(L, pbytes(L), vb, vb, vb));
    AMG_TRY((post_any<T, T, T, 0>(H, L, (const T*)L.b, (const T*)H->L[l + 1].x, (T*)L.x, q, s,
                                  nullptr, act, post_in(L, l))));
    PROF_END();
    AMG_TRY(post_sweeps(L, l, (T*)L.x));
  }
  const Level& L0 = H->L[0];
  const T* xc = (const T*)H->L[1].x;
  // one sweep: the dot products are fused into the post-smoother; several:
  // they follow the last sweep
  const bool smoothed = H->opt.smooth_prolongator != 0;
  const bool separate = L0.nu > 1 || smoothed;
  const int fused = separate ? 0 : dots;
  PROF_BEGIN(0, 2, bytes_post(L0, pbytes(L0), vb, 8.0, 8.0) + (fused > 1 ? 8.0 * L0.n : 0.0));
  const PostIn<T> in0 = post_in(L0, 0);
  int rc;
  if (fused == 0)
    rc = post_any<T, double, double, 0>(H, L0, r0, xc, z0, q, s, slice_part, act, in0);
  else if (fused == 1)
    rc = post_any<T, double, double, 1>(H, L0, r0, xc, z0, q, s, slice_part, act, in0);
  else
    rc = post_any<T, double, double, 2>(H, L0, r0, xc, z0, q, s, slice_part, act, in0);
  AMG_TRY(rc);
  PROF_END();
  if (L0.nu > 1) AMG_TRY(post_sweeps(L0, 0, z0));
  if (separate) AMG_TRY(separate_dots());
  return AMG_OK;
}

int vcycle_run(const amg_handle* H, const double* r, double* z, int dots, const double* q,
               cudaStream_t s, double* slice_part, const float* r32) {
  if (H->opt.precision == AMG_PREC_F32)
    return vcycle_levels<float>(H, r, z, dots, q, s, nullptr, slice_part, r32);
  return vcycle_levels<double>(H, r, z, dots, q, s, nullptr, slice_part);
}

// Device time of one pre- plus one post-smoothing pass of level l in its
// current layout (plus the FP64 SpMV of the PCG on level 0), averaged over
// `reps` after one warm-up.  b64/z64: FP64 level-0 vectors.
int time_level(const amg_handle* H, int l, int reps, const double* b64, double* z64, float* ms,
               cudaStream_t s) {
  const Level& L = H->L[l];
  const bool f32 = H->opt.precision == AMG_PREC_F32;
  auto once = [&]() -> int {
    if (!f32) {
      const double* b = l == 0 ? b64 : (const double*)L.b;
      double* x = l == 0 ? z64 : (double*)L.x;
      AMG_TRY((launch_pre<double, double, double>(H, L, L.ah64, b, (double*)L.r, s)));
      AMG_TRY((post_any<double, double, double, 0>(H, L, b, (const double*)H->L[l + 1].x, x,
                                                    nullptr, s)));
    } else if (l == 0) {
      AMG_TRY(pre_f32<double>(H, L, b64, (float*)L.r, s));
      AMG_TRY((post_any<float, double, double, 0>(H, L, b64, (const float*)H->L[1].x, z64,
                                                   nullptr, s)));
    } else {
      AMG_TRY(pre_f32<float>(H, L, (const float*)L.b, (float*)L.r, s));
      AMG_TRY((post_any<float, float, float, 0>(H, L, (const float*)L.b,
                                                 (const float*)H->L[l + 1].x, (float*)L.x,
                                                 nullptr, s)));
    }
    if (l == 0) AMG_TRY(sell_spmv64(L.A, 1.0, b64, 0.0, z64, H->num_sms, s));
    return AMG_OK;
  };
  cudaEvent_t e0, e1;
  AMG_CUDA_TRY(cudaEventCreate(&e0));
  AMG_CUDA_TRY(cudaEventCreate(&e1));
  int rc = once();
  if (rc == AMG_OK) rc = cudaEventRecord(e0, s) == cudaSuccess ? AMG_OK : AMG_ERR_CUDA;
  for (int k = 0; k < reps && rc == AMG_OK; ++k) rc = once();
  if (rc == AMG_OK) rc = cudaEventRecord(e1, s) == cudaSuccess ? AMG_OK : AMG_ERR_CUDA;
  if (rc == AMG_OK) rc = cudaEventSynchronize(e1) == cudaSuccess ? AMG_OK : AMG_ERR_CUDA;
  float t = 0.f;
  if (rc == AMG_OK) rc = cudaEventElapsedTime(&t, e0, e1) == cudaSuccess ? AMG_OK : AMG_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / (reps > 0 ? reps : 1);
  return rc;
}

int vcycle_profile(const amg_handle* H, const double* r, double* z, amg_kernel_time* out,
                   int max_out, int* count, cudaStream_t s) {
  Prof prof;
  prof.s = s;
  // An FP32 V-cycle inside PCG reads the FP32 copy of r that the CG update
  // writes; the profile does the same (the copy is made before, untimed).
  const float* r32 = nullptr;
  if (H->opt.precision == AMG_PREC_F32 && H->r32) {
    const int64_t n = H->L[0].n;
    k_vec_to_f32<<<grid_for(n, 256, H->num_sms, 8), 256, 0, s>>>(n, r, H->r32);
    AMG_LAUNCH_CHECK();
    r32 = H->r32;
  }
  // the level-0 post-smoother with the dot products PCG fuses into it: (r, z)
  // for FP64, (r, z) and (z, q) for the flexible FP32 form (q: scratch)
  const int dots = H->opt.precision == AMG_PREC_F32 ? 2 : 1;
  int rc = H->opt.precision == AMG_PREC_F32
               ? vcycle_levels<float>(H, r, z, dots, H->q, s, &prof, nullptr, r32)
               : vcycle_levels<double>(H, r, z, dots, H->q, s, &prof, nullptr);
  AMG_TRY(rc);
  AMG_TRY(prof.finish());
  const int m = (int)prof.rec.size();
  if (count) *count = m;
  for (int k = 0; k < m && k < max_out; ++k) out[k] = prof.rec[k];
  return AMG_OK;
}

int debug_convert(const double* in64, float* out32, const float* in32, double* out64,
                  int64_t n, cudaStream_t s) {
  if (n == 0) return AMG_OK;
  const int g = (int)std::min<int64_t>((n + 1023) / 1024, 4096);
  k_debug_convert<<<g, 256, 0, s>>>(n, in64, out32, in32, out64);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

}  // namespace amg
