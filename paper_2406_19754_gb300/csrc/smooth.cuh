// Per-row bodies of the V(1,1) cycle shared by the one-kernel-per-step path
// (vcycle.cu) and the persistent launch that runs the small levels between
// grid barriers (tail.cu).  Both call the same code, so a row's result is the
// same bits whichever kernel computes it.
//
//   pre_slice      r_i = b_i - (Ah b)_i                  (Ah = A S)
//   restrict_sum   b_c[I] = sum of r_i over the members of I, ascending
//   post_slice     z_i = s_i b_i + x_c[agg(i)] + s_i (r_i - (AP x_c)_i)
//   coarse_*       x = L^-T (L^-1 b) on a diagonal block of the coarsest level
//
// Ld picks the load path for vectors: LdRO (read-only cache) where no CTA of
// the launch writes them, LdL2 (L2-coherent) where another CTA of the same
// launch wrote them before a grid barrier, LdPlain where only the calling CTA
// wrote them before a __syncthreads.
#pragma once

#include "sellk.cuh"

namespace amg {

struct LdRO {
  template <typename X>
  __device__ __forceinline__ static X ld(const X* p) {
    return __ldg(p);
  }
};
// Plain loads: within one CTA, __syncthreads makes the CTA's own global
// writes visible to them (L1 stays coherent for the SM's own stores).
struct LdPlain {
  template <typename X>
  __device__ __forceinline__ static X ld(const X* p) {
    return *p;
  }
};
struct LdL2 {
  template <typename X>
  __device__ __forceinline__ static X ld(const X* p) {
    return __ldcg(p);
  }
};

// r_i = b_i - (Ah b)_i, accumulated from b_i down (negated FMAs: one FP64
// instruction an entry and none for the subtraction).
template <int TPR, typename Ld, typename V, typename T, typename BT>
__device__ __forceinline__ void pre_slice(const SellView<V>& Ah, const BT* b, T* r, int64_t sl,
                                          const Lanes<TPR>& ln) {
  const int64_t i = lane_row(Ah, sl, ln);
  const T bi = i >= 0 ? to_f(Ld::ld(b + i), T(0)) : T(0);
  const T acc = sell_row<TPR, T, true>(
      Ah, sl, ln, [&](int j) { return to_f(Ld::ld(b + j), T(0)); }, bi);
  if (i >= 0) r[i] = acc;
}

template <typename Ld, typename T>
__device__ __forceinline__ T restrict_sum(const int32_t* m, int stride, const T* r) {
  T acc = Ld::ld(r + m[0]);
  for (int k = 1; k < stride; ++k) {
    const int32_t i = m[k];
    if (i < 0) break;
    acc = acc + Ld::ld(r + i);
  }
  return acc;
}

// Writes x[i] = z_i for this lane's row and returns i (or -1, z untouched).
// xp: the pre-smoothed x when more than one sweep made it (else it is S b);
// e: if set, receives the residual b - A y of y = xp + P x_c, which further
// post-smoothing sweeps start from.
// One sweep (xp and e null): z_i = s_i (b_i + r_i - (AP x_c)_i) + x_c[agg(i)]
// (= S b + P x_c + S (r - AP x_c)), accumulated from b_i + r_i down with
// negated FMAs, then one FMA.
template <int TPR, typename Ld, typename V, typename T, typename BT, typename XT>
__device__ __forceinline__ int64_t post_slice(const SellView<V>& AP, const BT* b, const T* s,
                                              const T* r, const int32_t* agg, const T* xc, XT* x,
                                              int64_t sl, const Lanes<TPR>& ln, XT& z,
                                              const T* xp = nullptr, T* e = nullptr) {
  if (!xp && !e) {
    const int64_t i = lane_row(AP, sl, ln);
    const T init = i >= 0 ? to_f(Ld::ld(b + i), T(0)) + Ld::ld(r + i) : T(0);
    const T acc =
        sell_row<TPR, T, true>(AP, sl, ln, [&](int J) { return Ld::ld(xc + J); }, init);
    if (i >= 0) {
      z = to_f(fma(s[i], acc, Ld::ld(xc + agg[i])), XT(0));
      x[i] = z;
    }
    return i;
  }
  const T acc = sell_row<TPR, T>(AP, sl, ln, [&](int J) { return Ld::ld(xc + J); });
  const int64_t i = lane_row(AP, sl, ln);
  if (i >= 0) {
    // explicit FMAs: every kernel that runs this rounds identically
    const T si = s[i];
    const T xci = Ld::ld(xc + agg[i]);
    const T yi = xp ? Ld::ld(xp + i) + xci : fma(si, to_f(Ld::ld(b + i), T(0)), xci);
    const T ei = Ld::ld(r + i) - acc;
    z = to_f(fma(si, ei, yi), XT(0));
    x[i] = z;
    if (e) e[i] = ei;
  }
  return i;
}

// One step of the residual recurrence of an l1-Jacobi sweep: for r = b - A x,
// the sweep x' = x + S r leaves r' = r - (A S) r.  Gathers r through A S (one
// element per entry), writes r' to r_out, and hands back this lane's row i
// (-1 if none) with r_i and r'_i; the caller updates x (pre-smoother: x += S r,
// post-smoother, which steps the residual first: y += S r').
// The x updates of the sweeps, written out so every kernel rounds alike:
// pre-smoother x += S r (from x = S b on the first sweep), post-smoother
// y += S r' (y possibly wider than the V-cycle type).
template <typename T>
__device__ __forceinline__ T sweep_pre_x(T xi, T si, T ri) {
  return fma(si, ri, xi);
}
template <typename T, typename YT>
__device__ __forceinline__ YT sweep_post_y(YT yi, T si, T rn) {
  if constexpr (sizeof(YT) == sizeof(T))
    return fma(si, rn, yi);
  else
    return yi + to_f(si * rn, YT(0));
}

template <int TPR, typename Ld, typename V, typename T>
__device__ __forceinline__ void sweep_slice(const SellView<V>& Ah, const T* s, const T* r,
                                            T* r_out, int64_t sl, const Lanes<TPR>& ln,
                                            T& ri, T& rn, int64_t& i) {
  const T acc = sell_row<TPR, T>(Ah, sl, ln, [&](int j) { return Ld::ld(r + j); });
  i = lane_row(Ah, sl, ln);
  if (i >= 0) {
    ri = Ld::ld(r + i);
    rn = ri - acc;
    r_out[i] = rn;
  }
}

// One diagonal block of the coarsest level solved by the calling CTA:
// y = L^-1 b, then x = L^-T y, one warp per row, vectors staged in shared
// memory (2n doubles).  Every thread of the CTA must call it.
template <typename Ld, typename BT, typename XT>
__device__ __forceinline__ void coarse_block_solve(int blk, const int64_t* brow,
                                                   const int64_t* bmat, const double* Linv_all,
                                                   const double* LinvT_all, const BT* b_all,
                                                   XT* x_all, double* csh) {
  const int64_t r0 = brow[blk];
  const int n = (int)(brow[blk + 1] - r0);
  const double* Linv = Linv_all + bmat[blk];
  const double* LinvT = LinvT_all + bmat[blk];
  const BT* b = b_all + r0;
  XT* x = x_all + r0;
  double* bs = csh;
  double* ys = csh + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) bs[i] = (double)Ld::ld(b + i);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = w; i < n; i += nw) {
    double acc = 0.0;
    const double* row = Linv + (int64_t)i * n;
    for (int k = lane; k <= i; k += 32) acc = fma(row[k], bs[k], acc);
    acc = warp_sum(acc);
    if (lane == 0) ys[i] = acc;
  }
  __syncthreads();
  for (int k = w; k < n; k += nw) {
    double acc = 0.0;
    const double* row = LinvT + (int64_t)k * n;
    for (int i = k + lane; i < n; i += 32) acc = fma(row[i], ys[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) x[k] = (XT)acc;
  }
  __syncthreads();  // bs/ys are reused by the CTA's next block
}

// Large coarsest blocks: row g of y = L^-1 b and of x = L^-T y, one warp
// each.  Each dot product is summed like coarse_block_solve sums it (lane
// partials over a stride of 32, then the xor tree), so results agree bit for
// bit.
template <typename Ld, typename BT>
__device__ __forceinline__ void coarse_y_row(int64_t g, int nblk, const int64_t* brow,
                                             const int64_t* bmat, const double* Linv_all,
                                             const BT* b, double* y) {
  const int lane = threadIdx.x & 31;
  const int blk = coarse_block(brow, nblk, g);
  const int64_t r0 = brow[blk];
  const int64_t n = brow[blk + 1] - r0, i = g - r0;
  const double* row = Linv_all + bmat[blk] + i * n;
  double acc = 0.0;
  for (int64_t k = lane; k <= i; k += 32) acc = fma(row[k], (double)Ld::ld(b + r0 + k), acc);
  acc = warp_sum(acc);
  if (lane == 0) y[g] = acc;
}

template <typename Ld, typename XT>
__device__ __forceinline__ void coarse_x_row(int64_t g, int nblk, const int64_t* brow,
                                             const int64_t* bmat, const double* LinvT_all,
                                             const double* y, XT* x) {
  const int lane = threadIdx.x & 31;
  const int blk = coarse_block(brow, nblk, g);
  const int64_t r0 = brow[blk];
  const int64_t n = brow[blk + 1] - r0, k = g - r0;
  const double* row = LinvT_all + bmat[blk] + k * n;
  double acc = 0.0;
  for (int64_t i = k + lane; i < n; i += 32) acc = fma(row[i], Ld::ld(y + r0 + i), acc);
  acc = warp_sum(acc);
  if (lane == 0) x[g] = (XT)acc;
}

// Coarsest solve by PCG with the l1-Jacobi preconditioner (s = 1/d of the
// coarsest level; Sec. 3, the VBM/VMATCH coarsest solver), zero initial guess,
// in one CUDA block: at most maxit iterations, stopping once ||r|| <= tol ||b||
// or when p^T A p <= 0.  FP64 throughout; dot products by a fixed block tree.
// w: 5n doubles of scratch (x, r, z, p, q).  Every thread of the block calls
// it; b may have been written by the same block before a __syncthreads.
__device__ __forceinline__ double block_dot(int64_t n, const double* u, const double* v) {
  __shared__ double total;
  double t[1] = {0.0};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) t[0] += u[i] * v[i];
  block_sum<1>(t);
  if (threadIdx.x == 0) total = t[0];
  __syncthreads();
  const double res = total;
  __syncthreads();
  return res;
}

template <int TPR, typename BT, typename XT>
__device__ void coarse_pcg_cta(const SellView<double>& A, const double* sinv, const BT* b,
                               XT* xo, double* w, int maxit, double tol) {
  const int64_t n = A.n;
  double* x = w;
  double* r = w + n;
  double* z = w + 2 * n;
  double* p = w + 3 * n;
  double* q = w + 4 * n;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    x[i] = 0.0;
    r[i] = (double)b[i];
  }
  __syncthreads();
  const double bnorm = sqrt(block_dot(n, r, r));
  if (bnorm > 0.0) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      z[i] = sinv[i] * r[i];
      p[i] = z[i];
    }
    __syncthreads();
    double rz = block_dot(n, r, z);
    const Lanes<TPR> ln;
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int k = 0; k < maxit; ++k) {
      for (int64_t sl = warp; sl < A.ngroups; sl += nwarps) {
        const double acc = sell_row<TPR, double>(A, sl, ln, [&](int j) { return p[j]; });
        const int64_t i = lane_row(A, sl, ln);
        if (i >= 0) q[i] = acc;
      }
      __syncthreads();
      const double pq = block_dot(n, p, q);
      if (!(pq > 0.0)) break;
      const double alpha = rz / pq;
      // x, r, z and the sums (r, r), (r, z) in one pass: each thread adds the
      // rows it updates, in the order block_dot would, so the sums are the
      // same bits as two separate block_dot calls
      double t[2] = {0.0, 0.0};
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        x[i] = x[i] + alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        const double zi = sinv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        t[0] += ri * ri;
        t[1] += ri * zi;
      }
      block_sum<2>(t);
      __shared__ double rr_rz[2];
      if (threadIdx.x == 0) {
        rr_rz[0] = t[0];
        rr_rz[1] = t[1];
      }
      __syncthreads();
      const double rr = rr_rz[0], rzn = rr_rz[1];
      if (sqrt(rr) <= tol * bnorm) break;
      const double beta = rzn / rz;
      for (int64_t i = threadIdx.x; i < n; i += blockDim.x) p[i] = z[i] + beta * p[i];
      __syncthreads();
      rz = rzn;
    }
  }
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) xo[i] = bnorm > 0.0 ? (XT)x[i] : XT(0);
}

}  // namespace amg
