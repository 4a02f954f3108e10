// Sparse products for the smoothed prolongator (Sec. 2.3): C = X Y for CSR
// X (n x m) and Y (m x k) with ascending columns in every row, and the
// transpose of a CSR matrix.
//
// One warp builds one row of C.  It walks row i of X in order; for entry
// (i, k) the lanes take the entries of row k of Y (distinct columns, so no
// two lanes touch the same output) and add x_ik * y_kJ into a per-warp hash
// table in shared memory.  Every output entry therefore sums its
// contributions in ascending order of the inner index, one correctly rounded
// product and one correctly rounded addition each (no fused multiply-add),
// the first contribution starting the sum: the same bits as a sequential
// loop.  A first pass counts each row's distinct columns; the second fills
// values and writes the columns in ascending order.  Rows with more than
// SPG_LARGE distinct columns are reported (AMG_ERR_UNSUPPORTED).
#include <string.h>

#include <algorithm>

#include "common.cuh"

namespace amg {

namespace {

// Rows go to one warp with a small table first; rows with more distinct
// columns than it holds are listed and redone by one warp per block with a
// large table (coarse levels of a smoothed hierarchy reach a few hundred
// columns per row).
constexpr int SPG_SMALL = 512;   // slots of a small table
constexpr int SPG_LARGE = 8192;  // slots of a large table (115 KB of shared memory)
constexpr int SPG_WARPS = 4;     // warps (small tables) per block
constexpr int32_t SPG_EMPTY = -1;

template <int SLOTS>
__device__ __forceinline__ int spg_hash(int32_t J) {
  constexpr int LOG = SLOTS == 512 ? 9 : 13;
  static_assert((1 << LOG) == SLOTS, "table size");
  return (int)(((uint32_t)J * 2654435761u) >> (32 - LOG));
}

// Slot of column J (inserted if new); -1 when the table is full.
template <int SLOTS>
__device__ __forceinline__ int spg_slot(int32_t* keys, int32_t J, int* used) {
  int h = spg_hash<SLOTS>(J);
  for (int probe = 0; probe < SLOTS; ++probe) {
    const int32_t k = keys[h];
    if (k == J) return h;
    if (k == SPG_EMPTY) {
      const int32_t prev = atomicCAS(&keys[h], SPG_EMPTY, J);
      if (prev == SPG_EMPTY) {
        atomicAdd(used, 1);
        return h;
      }
      if (prev == J) return h;
    }
    h = (h + 1) & (SLOTS - 1);
  }
  return -1;
}

template <bool FILL, int SLOTS>
constexpr size_t spg_smem(int warps) {
  return (size_t)warps * (SLOTS * (4 + (FILL ? 8 + 2 : 0)) + 8);
}

// FILL = false: cnt[i] = distinct columns of row i.  FILL = true: writes the
// row's columns (ascending) and sums at C_rp[i].  Sums start from -0.0, which
// leaves the first contribution unchanged (-0 + t = t for every t).
// rows: the rows to build (null: all n); a small-table launch skips rows
// whose count exceeds its table and, when counting, lists them in big.
template <bool FILL, int SLOTS>
__global__ void k_spgemm(int64_t n, const int64_t* __restrict__ rows,
                         const int64_t* __restrict__ X_rp, const int32_t* __restrict__ X_ci,
                         const double* __restrict__ X_v, const int64_t* __restrict__ Y_rp,
                         const int32_t* __restrict__ Y_ci, const double* __restrict__ Y_v,
                         int64_t* cnt, int64_t* big, unsigned long long* nbig,
                         const int64_t* __restrict__ C_rp, int32_t* __restrict__ C_ci,
                         double* __restrict__ C_v, int* status) {
  extern __shared__ __align__(16) unsigned char spg_sh[];
  const int warps = blockDim.x >> 5;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per warp: vals (FILL), keys, list (FILL), used
  unsigned char* base = spg_sh + (size_t)w * (SLOTS * (4 + (FILL ? 8 + 2 : 0)) + 8);
  double* vals = (double*)base;
  int32_t* keys = (int32_t*)(base + (FILL ? 8 * SLOTS : 0));
  int16_t* list = (int16_t*)(base + (FILL ? 12 * SLOTS : 0));
  int* used = (int*)(base + SLOTS * (4 + (FILL ? 8 + 2 : 0)));
  const int64_t nw = (int64_t)gridDim.x * warps;
  for (int64_t t = (int64_t)blockIdx.x * warps + w; t < n; t += nw) {
    const int64_t i = rows ? rows[t] : t;
    if (FILL && !rows && C_rp[i + 1] - C_rp[i] > SLOTS) continue;  // a large-table row
    for (int s = lane; s < SLOTS; s += 32) {
      keys[s] = SPG_EMPTY;
      if (FILL) vals[s] = -0.0;
    }
    if (lane == 0) *used = 0;
    __syncwarp();
    bool full = false;
    for (int64_t e = X_rp[i]; e < X_rp[i + 1]; ++e) {
      const int32_t k = X_ci[e];
      const double xv = FILL ? X_v[e] : 0.0;
      for (int64_t f = Y_rp[k] + lane; f < Y_rp[k + 1]; f += 32) {
        const int h = spg_slot<SLOTS>(keys, Y_ci[f], used);
        if (h < 0) {
          full = true;
          continue;
        }
        if (FILL) vals[h] = __dadd_rn(vals[h], __dmul_rn(xv, Y_v[f]));
      }
      __syncwarp();  // the next inner index sees this one's sums
    }
    full = __any_sync(0xffffffffu, full);
    if (full) {
      if (lane == 0) {
        if (big) {
          big[atomicAdd(nbig, 1ull)] = i;
        } else {
          atomicExch(status, AMG_ERR_UNSUPPORTED);
        }
      }
      __syncwarp();
      continue;
    }
    if (!FILL) {
      if (lane == 0) cnt[i] = *used;
      __syncwarp();
      continue;
    }
    // compact the used slots, then place each at the rank of its column
    int m = 0;
    for (int s0 = 0; s0 < SLOTS; s0 += 32) {
      const bool u = keys[s0 + lane] != SPG_EMPTY;
      const unsigned b = __ballot_sync(0xffffffffu, u);
      if (u) list[m + __popc(b & ((1u << lane) - 1u))] = (int16_t)(s0 + lane);
      m += __popc(b);
    }
    __syncwarp();
    const int64_t c0 = C_rp[i];
    for (int a = lane; a < m; a += 32) {
      const int32_t J = keys[list[a]];
      int rank = 0;
      for (int u = 0; u < m; ++u) rank += keys[list[u]] < J ? 1 : 0;
      C_ci[c0 + rank] = J;
      C_v[c0 + rank] = vals[list[a]];
    }
    __syncwarp();
  }
}

// Transpose: entries scattered by an atomic cursor per column, then every
// row of the transpose sorted by column (its source rows are distinct), so
// the result does not depend on the scatter order.
__global__ void k_tr_count(int64_t nnz, const int32_t* __restrict__ ci, int64_t* cnt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd((unsigned long long*)&cnt[ci[e]], 1ull);
}

__global__ void k_tr_fill(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ v, int64_t* cursor, int32_t* T_ci,
                          double* T_v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int64_t p = (int64_t)atomicAdd((unsigned long long*)&cursor[ci[e]], 1ull);
      T_ci[p] = (int32_t)i;
      T_v[p] = v[e];
    }
}

// Sorts the entries of every row by column (insertion sort: short rows).
__global__ void k_sort_rows(int64_t n, const int64_t* __restrict__ rp, int32_t* ci, double* v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t e = rp[i] + 1; e < rp[i + 1]; ++e) {
      const int32_t c = ci[e];
      const double x = v[e];
      int64_t f = e - 1;
      while (f >= rp[i] && ci[f] > c) {
        ci[f + 1] = ci[f];
        v[f + 1] = v[f];
        --f;
      }
      ci[f + 1] = c;
      v[f + 1] = x;
    }
}

// w = 1 / max_i (sum_j |a_ij|) / a_ii: the row ratios are non-negative, so
// their bit patterns order like the values and an integer maximum is exact.
__global__ void k_ratio_max(int64_t n, const int64_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, const double* __restrict__ v,
                            unsigned long long* out) {
  unsigned long long best = 0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0, d = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      s = __dadd_rn(s, fabs(v[e]));
      if (ci[e] == i) d = v[e];
    }
    const unsigned long long b = (unsigned long long)__double_as_longlong(__ddiv_rn(s, d));
    best = b > best ? b : best;
  }
  atomicMax(out, best);
}

// In place: (A P_hat)_iJ -> P_iJ = [agg(i) = J] - w ((A P_hat)_iJ / a_ii), then
// the row's columns ascending.
__global__ void k_smooth_p(int64_t n, const int64_t* __restrict__ A_rp,
                           const int32_t* __restrict__ A_ci, const double* __restrict__ A_v,
                           const int32_t* __restrict__ agg, const int64_t* __restrict__ rp,
                           int32_t* ci, double* v, double w) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double aii = 0.0;
    for (int64_t e = A_rp[i]; e < A_rp[i + 1]; ++e)
      if (A_ci[e] == i) aii = A_v[e];
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const double ind = ci[e] == agg[i] ? 1.0 : 0.0;
      v[e] = __dsub_rn(ind, __dmul_rn(w, __ddiv_rn(v[e], aii)));
    }
    for (int64_t e = rp[i] + 1; e < rp[i + 1]; ++e) {
      const int32_t c = ci[e];
      const double x = v[e];
      int64_t f = e - 1;
      while (f >= rp[i] && ci[f] > c) {
        ci[f + 1] = ci[f];
        v[f + 1] = v[f];
        --f;
      }
      ci[f + 1] = c;
      v[f + 1] = x;
    }
  }
}

// A_F for the filtered prolongator smoothing: the diagonal and the entries
// with |a_ij| >= theta sqrt(a_ii a_jj) kept, the dropped ones of each row
// added (in stored order) to its diagonal.
__device__ __forceinline__ bool filter_drop(int64_t i, int32_t j, double v,
                                            const double* __restrict__ diag, double theta) {
  return j != i && !(fabs(v) >= __dmul_rn(theta, __dsqrt_rn(__dmul_rn(diag[i], diag[j]))));
}

__global__ void k_filter_count(int64_t n, const int64_t* __restrict__ rp,
                               const int32_t* __restrict__ ci, const double* __restrict__ va,
                               const double* __restrict__ diag, double theta, int64_t* cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = 0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
      if (!filter_drop(i, ci[e], va[e], diag, theta)) ++c;
    cnt[i] = c;
  }
}

__global__ void k_filter_fill(int64_t n, const int64_t* __restrict__ rp,
                              const int32_t* __restrict__ ci, const double* __restrict__ va,
                              const double* __restrict__ diag, double theta,
                              const int64_t* __restrict__ frp, int32_t* __restrict__ fci,
                              double* __restrict__ fva) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double lump = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
      if (filter_drop(i, ci[e], va[e], diag, theta)) lump = __dadd_rn(lump, va[e]);
    int64_t pos = frp[i];
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int32_t j = ci[e];
      if (filter_drop(i, j, va[e], diag, theta)) continue;
      fci[pos] = j;
      fva[pos] = j == i ? __dadd_rn(va[e], lump) : va[e];
      ++pos;
    }
  }
}

}  // namespace

int filter_matrix(Arena& ar, int64_t n, const int64_t* rp, const int32_t* ci, const double* va,
                  const double* diag, double theta, int64_t** F_rp, int32_t** F_ci,
                  double** F_v, int num_sms, cudaStream_t s) {
  int64_t* cnt = nullptr;
  AMG_TRY(ar.alloc_n(&cnt, n + 1));
  AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (n + 1), s));
  const int g = grid_for(n, 256, num_sms, 8);
  k_filter_count<<<g, 256, 0, s>>>(n, rp, ci, va, diag, theta, cnt);
  AMG_LAUNCH_CHECK();
  AMG_TRY(ar.alloc_n(F_rp, n + 1));
  int64_t total = 0;
  AMG_TRY(scan_exclusive_i64(ar, cnt, *F_rp, n + 1, &total, s));
  ar.release(cnt);
  AMG_TRY(ar.alloc_n(F_ci, total > 0 ? total : 1));
  AMG_TRY(ar.alloc_n(F_v, total > 0 ? total : 1));
  k_filter_fill<<<g, 256, 0, s>>>(n, rp, ci, va, diag, theta, *F_rp, *F_ci, *F_v);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

int spgemm(Arena& ar, int64_t n, const int64_t* X_rp, const int32_t* X_ci, const double* X_v,
           const int64_t* Y_rp, const int32_t* Y_ci, const double* Y_v, int64_t** C_rp,
           int32_t** C_ci, double** C_v, int64_t* C_nnz, int* dev_status, int num_sms,
           cudaStream_t s) {
  constexpr size_t sm_cs = spg_smem<false, SPG_SMALL>(SPG_WARPS);
  constexpr size_t sm_fs = spg_smem<true, SPG_SMALL>(SPG_WARPS);
  constexpr size_t sm_cl = spg_smem<false, SPG_LARGE>(1);
  constexpr size_t sm_fl = spg_smem<true, SPG_LARGE>(1);
  AMG_CUDA_TRY(cudaFuncSetAttribute(k_spgemm<true, SPG_LARGE>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fl));
  int64_t* cnt = nullptr;
  int64_t* big = nullptr;
  unsigned long long* nbig_d = nullptr;
  AMG_TRY(ar.alloc_n(&cnt, n + 1));
  AMG_TRY(ar.alloc_n(&big, n > 0 ? n : 1));
  AMG_TRY(ar.alloc_n(&nbig_d, 1));
  AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (n + 1), s));
  AMG_CUDA_TRY(cudaMemsetAsync(nbig_d, 0, sizeof(*nbig_d), s));
  const int grid = grid_for(n, SPG_WARPS, num_sms, 16);
  k_spgemm<false, SPG_SMALL><<<grid, 32 * SPG_WARPS, sm_cs, s>>>(
      n, nullptr, X_rp, X_ci, X_v, Y_rp, Y_ci, Y_v, cnt, big, nbig_d, nullptr, nullptr, nullptr,
      dev_status);
  AMG_LAUNCH_CHECK();
  unsigned long long nbig = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&nbig, nbig_d, sizeof(nbig), cudaMemcpyDeviceToHost, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  const int gbig = grid_for((int64_t)nbig, 1, num_sms, 4);
  if (nbig > 0) {
    k_spgemm<false, SPG_LARGE><<<gbig, 32, sm_cl, s>>>(
        (int64_t)nbig, big, X_rp, X_ci, X_v, Y_rp, Y_ci, Y_v, cnt, nullptr, nullptr, nullptr,
        nullptr, nullptr, dev_status);
    AMG_LAUNCH_CHECK();
  }
  AMG_TRY(ar.alloc_n(C_rp, n + 1));
  int64_t total = 0;
  AMG_TRY(scan_exclusive_i64(ar, cnt, *C_rp, n + 1, &total, s));
  ar.release(cnt);
  *C_nnz = total;
  AMG_TRY(ar.alloc_n(C_ci, total > 0 ? total : 1));
  AMG_TRY(ar.alloc_n(C_v, total > 0 ? total : 1));
  k_spgemm<true, SPG_SMALL><<<grid, 32 * SPG_WARPS, sm_fs, s>>>(
      n, nullptr, X_rp, X_ci, X_v, Y_rp, Y_ci, Y_v, nullptr, nullptr, nullptr, *C_rp, *C_ci, *C_v,
      dev_status);
  AMG_LAUNCH_CHECK();
  if (nbig > 0) {
    k_spgemm<true, SPG_LARGE><<<gbig, 32, sm_fl, s>>>(
        (int64_t)nbig, big, X_rp, X_ci, X_v, Y_rp, Y_ci, Y_v, nullptr, nullptr, nullptr, *C_rp,
        *C_ci, *C_v, dev_status);
    AMG_LAUNCH_CHECK();
  }
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  ar.release(big);
  ar.release(nbig_d);
  return AMG_OK;
}

int transpose_csr(Arena& ar, int64_t n, int64_t ncols, const int64_t* rp, const int32_t* ci,
                  const double* v, int64_t nnz, int64_t** T_rp, int32_t** T_ci, double** T_v,
                  int num_sms, cudaStream_t s) {
  int64_t* cnt = nullptr;
  AMG_TRY(ar.alloc_n(&cnt, ncols + 1));
  AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (ncols + 1), s));
  k_tr_count<<<grid_for(nnz, 256, num_sms, 8), 256, 0, s>>>(nnz, ci, cnt);
  AMG_LAUNCH_CHECK();
  AMG_TRY(ar.alloc_n(T_rp, ncols + 1));
  int64_t total = 0;
  AMG_TRY(scan_exclusive_i64(ar, cnt, *T_rp, ncols + 1, &total, s));
  AMG_CUDA_TRY(cudaMemcpyAsync(cnt, *T_rp, sizeof(int64_t) * ncols, cudaMemcpyDeviceToDevice, s));
  AMG_TRY(ar.alloc_n(T_ci, nnz));
  AMG_TRY(ar.alloc_n(T_v, nnz));
  k_tr_fill<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(n, rp, ci, v, cnt, *T_ci, *T_v);
  AMG_LAUNCH_CHECK();
  k_sort_rows<<<grid_for(ncols, 256, num_sms, 8), 256, 0, s>>>(ncols, *T_rp, *T_ci, *T_v);
  AMG_LAUNCH_CHECK();
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  ar.release(cnt);
  return AMG_OK;
}

int smoothed_prolongator(Arena& ar, int64_t n, const int64_t* A_rp, const int32_t* A_ci,
                         const double* A_v, const int32_t* agg, const int64_t* rp, int32_t* ci,
                         double* v, double* w_out, int num_sms, cudaStream_t s) {
  unsigned long long* m = nullptr;
  AMG_TRY(ar.alloc_n(&m, 1));
  AMG_CUDA_TRY(cudaMemsetAsync(m, 0, sizeof(*m), s));
  k_ratio_max<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(n, A_rp, A_ci, A_v, m);
  AMG_LAUNCH_CHECK();
  unsigned long long bits = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&bits, m, sizeof(bits), cudaMemcpyDeviceToHost, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  ar.release(m);
  double ratio;
  memcpy(&ratio, &bits, sizeof(ratio));
  const double w = 1.0 / ratio;
  *w_out = w;
  k_smooth_p<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(n, A_rp, A_ci, A_v, agg, rp, ci, v, w);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

}  // namespace amg
