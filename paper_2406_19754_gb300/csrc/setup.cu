// Hierarchy setup on the GPU (Sec. 2.3): l1-Jacobi diagonal, pairwise
// locally-dominant weighted matching, aggregate numbering, the Galerkin
// product A_{l+1} = P^T A_l P with a piecewise-constant 0/1 P, and the dense
// Cholesky factor of the coarsest level.
//
// Bit-exactness: every value the setup produces (matching weights, Galerkin
// sums, l1 row sums, Cholesky factor) is computed with explicitly rounded
// operations (__dadd_rn, __dmul_rn, ...) in a fixed order, so no FMA
// contraction can change a bit, and the aggregates and coarse matrices are
// reproducible run to run and against a sequential FP64 evaluation in the
// same order.
#include <algorithm>
#include <map>
#include <mutex>

#include "common.cuh"
#include "sellk.cuh"

namespace amg {

// ------------------------------------------------------------------ l1 diagonal

// d_i = sum_j |a_ij| in stored (ascending column) order; diag_i = a_ii.
__global__ void k_l1_diag(int64_t n, const int64_t* rowptr, const int32_t* col,
                          const double* val, double* d, double* diag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0, a = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      double v = val[e];
      s = __dadd_rn(s, fabs(v));
      if (col[e] == i) a = v;
    }
    if (d) d[i] = s;
    diag[i] = a;
  }
}

// s_i = omega_i * (1 / d_i) (omega == NULL: 1).
// 1 / d_i, once per level at setup (an FP64 division is a long sequence on
// GB300's reduced-rate FP64 pipe; new smoother weights only multiply).
__global__ void k_recip(int64_t n, const double* d, double* dinv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dinv[i] = __ddiv_rn(1.0, d[i]);
}

// s_i = omega_i * (1 / d_i) (omega == 1 when null).
__global__ void k_smoother_scale(int64_t n, const double* dinv, const float* omega, double* s64,
                                 float* s32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double inv = dinv[i];
    double w = omega ? (double)omega[i] : 1.0;
    double s = __dmul_rn(w, inv);
    s64[i] = s;
    if (s32) s32[i] = (float)s;
  }
}

// ------------------------------------------------------------------ matching
// Edge weight (compatible weighted matching, w == 1):
//   c_ij = 1 - (2 a_ij) / (a_ii + a_jj);  eligible iff c_ij > 0.
// Strict total order on edges: (c, -lo, -hi), larger wins, i.e. equal weights
// go to the edge with the smaller endpoints (the order of a sequential greedy
// pass over the rows).  Locally-dominant rounds: every active vertex points
// at its heaviest eligible unmatched neighbour; mutual pointers match.  Under
// a strict total order this reproduces greedy matching in descending key
// order exactly.
//
// Only vertices whose neighbourhood changed need a new pointer, so each round
// works on a frontier list: the unmatched neighbours of the vertices matched
// in the previous round.  Total work is O(nnz) however many rounds the
// dependency chains need (on lexicographically numbered grids the index
// order makes them a diagonal wavefront of ~2.5 x side rounds).

struct EdgeKey {
  double c;
  int32_t lo, hi;
};

__device__ __forceinline__ bool heavier(const EdgeKey& a, const EdgeKey& b) {
  if (a.c != b.c) return a.c > b.c;
  if (a.lo != b.lo) return a.lo < b.lo;
  return a.hi < b.hi;
}

// mate[i]: >= 0 matched, -1 active, -2 no eligible partner left (singleton).
// flag[i]: 1 while i sits on the next frontier list.
__global__ void k_match_cand(const int32_t* __restrict__ wl, const int* __restrict__ nwl,
                             const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ diag,
                             const int32_t* __restrict__ mate, int32_t* __restrict__ cand,
                             int32_t* __restrict__ flag, int* rounds) {
  const int nw = *nwl;
  if (blockIdx.x == 0 && threadIdx.x == 0 && nw > 0) ++*rounds;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nw; t += gridDim.x * blockDim.x) {
    const int32_t i = wl[t];
    flag[i] = 0;
    if (mate[i] != -1) continue;
    const double di = diag[i];
    EdgeKey best;
    int32_t bj = -1;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int32_t j = col[e];
      if (j == i || mate[j] != -1) continue;
      double a;
      if (!edge_value(rowptr, col, val, i, j, val[e], &a)) continue;
      const double c = __dsub_rn(1.0, __ddiv_rn(__dmul_rn(2.0, a), __dadd_rn(di, diag[j])));
      if (!(c > 0.0)) continue;
      EdgeKey k;
      k.c = c;
      k.lo = min(j, i);
      k.hi = max(j, i);
      if (bj < 0 || heavier(k, best)) {
        best = k;
        bj = j;
      }
    }
    cand[i] = bj;
  }
}

// Mutual pointers match; a vertex without an eligible neighbour is final.
__global__ void k_match_commit(const int32_t* __restrict__ wl, const int* __restrict__ nwl,
                               const int32_t* __restrict__ cand, int32_t* mate) {
  const int nw = *nwl;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nw; t += gridDim.x * blockDim.x) {
    const int32_t i = wl[t];
    if (mate[i] != -1) continue;
    const int32_t j = cand[i];
    if (j < 0) {
      mate[i] = -2;
    } else if (cand[j] == i) {  // both sides may write: same values
      mate[i] = j;
      mate[j] = i;
    }
  }
}

// Next frontier: unmatched neighbours of the pairs matched in this round.
__global__ void k_match_expand(const int32_t* __restrict__ wl, const int* __restrict__ nwl,
                               const int64_t* __restrict__ rowptr,
                               const int32_t* __restrict__ col, const int32_t* __restrict__ mate,
                               int32_t* __restrict__ flag, int32_t* __restrict__ wl_next,
                               int* __restrict__ nwl_next) {
  const int nw = *nwl;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nw; t += gridDim.x * blockDim.x) {
    const int32_t i = wl[t];
    const int32_t m = mate[i];
    if (m < 0) continue;  // frontier vertices were unmatched when the round began
    for (int side = 0; side < 2; ++side) {
      const int32_t v = side == 0 ? i : m;
      for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
        const int32_t k = col[e];
        if (k != v && mate[k] == -1 && atomicExch(&flag[k], 1) == 0)
          wl_next[atomicAdd(nwl_next, 1)] = k;
      }
    }
  }
}

__global__ void k_match_final(int64_t n, int32_t* mate) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (mate[i] < 0) mate[i] = -1;
}

__global__ void k_match_counts(int* cnt, int n) {
  if (threadIdx.x == 0) {
    cnt[0] = n;  // the first frontier holds every row
    cnt[1] = 0;
    cnt[2] = 0;  // rounds with a non-empty frontier
    cnt[3] = 0;
  }
}

// The rounds of locally-dominant matching on caller-provided scratch: cand
// and flag hold n entries, wl two frontiers of n entries at wl and
// wl + wl_stride, cnt 4 ints.  Every entry point that matches runs this loop,
// so they launch the same kernels in the same order.
int match_round_loop(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                     const double* diag, int32_t* mate, int32_t* cand, int32_t* flag,
                     int32_t* wl, int64_t wl_stride, int* cnt, int* rounds_out, int num_sms,
                     cudaStream_t s) {
  // scratch may hold an earlier call's contents: reset what must start at zero
  AMG_CUDA_TRY(cudaMemsetAsync(mate, 0xFF, sizeof(int32_t) * n, s));
  AMG_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int32_t) * n, s));
  const int grid = grid_for(n, 256, num_sms, 8);
  k_match_counts<<<1, 32, 0, s>>>(cnt, (int)n);
  AMG_LAUNCH_CHECK();
  k_iota<<<grid, 256, 0, s>>>(n, wl);
  AMG_LAUNCH_CHECK();
  int cur = 0;
  int rc = AMG_OK;
  int64_t launched = 0;
  for (;;) {
    // a batch of rounds between host checks; empty rounds exit immediately
    for (int r = 0; r < 8; ++r) {
      int32_t* w = wl + (int64_t)cur * wl_stride;
      int32_t* wn = wl + (int64_t)(1 - cur) * wl_stride;
      k_match_cand<<<grid, 256, 0, s>>>(w, cnt + cur, rowptr, col, val, diag, mate, cand, flag,
                                        cnt + 2);
      AMG_LAUNCH_CHECK();
      k_match_commit<<<grid, 256, 0, s>>>(w, cnt + cur, cand, mate);
      AMG_LAUNCH_CHECK();
      AMG_CUDA_TRY(cudaMemsetAsync(cnt + 1 - cur, 0, sizeof(int), s));
      k_match_expand<<<grid, 256, 0, s>>>(w, cnt + cur, rowptr, col, mate, flag, wn,
                                          cnt + 1 - cur);
      AMG_LAUNCH_CHECK();
      cur = 1 - cur;
    }
    launched += 8;
    int h[4];
    AMG_CUDA_TRY(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (h[cur] == 0) {
      if (rounds_out) *rounds_out = h[2];
      break;
    }
    if (launched > 4 * n + 64) {  // each round matches at least the heaviest edge
      rc = AMG_ERR_DEVICE_CHECK;
      break;
    }
  }
  k_match_final<<<grid, 256, 0, s>>>(n, mate);
  AMG_LAUNCH_CHECK();
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  return rc;
}

static int match_rounds(Arena& ar, int64_t n, const int64_t* rowptr, const int32_t* col,
                        const double* val, const double* diag, int32_t* mate, int* rounds_out,
                        int num_sms, cudaStream_t s) {
  int32_t *cand = nullptr, *flag = nullptr, *wl = nullptr;
  int* cnt = nullptr;  // [0], [1]: frontier sizes; [2]: rounds with a non-empty frontier
  AMG_TRY(ar.alloc_n(&cand, n));
  AMG_TRY(ar.alloc_n(&flag, n));
  AMG_TRY(ar.alloc_n(&wl, 2 * n));
  AMG_TRY(ar.alloc_n(&cnt, 4));
  const int rc = match_round_loop(n, rowptr, col, val, diag, mate, cand, flag, wl, n, cnt,
                                  rounds_out, num_sms, s);
  ar.release(cand);
  ar.release(flag);
  ar.release(wl);
  ar.release(cnt);
  return rc;
}

int match_pairwise(Arena& ar, int64_t n, const int64_t* rowptr, const int32_t* col,
                   const double* val, int32_t* mate, int* rounds, cudaStream_t s) {
  int dev = 0, sms = 0;
  AMG_CUDA_TRY(cudaGetDevice(&dev));
  AMG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double* diag = nullptr;
  AMG_TRY(ar.alloc_n(&diag, n));
  k_l1_diag<<<grid_for(n, 256, sms, 8), 256, 0, s>>>(n, rowptr, col, val, nullptr, diag);
  AMG_LAUNCH_CHECK();
  int rc = match_rounds(ar, n, rowptr, col, val, diag, mate, rounds, sms, s);
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  ar.release(diag);
  return rc;
}

// ------------------------------------------------------------------ aggregation

__global__ void k_leader_flags(int64_t n, const int32_t* mate, int32_t* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t m = mate[i];
    flag[i] = (m < 0 || m > i) ? 1 : 0;
  }
}

// agg of a pair is the number of its smaller member; composes comp = agg[comp].
__global__ void k_assign_compose(int64_t n_fine, int64_t n, const int32_t* mate,
                                 const int32_t* id, int32_t* comp) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n_fine;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = comp[f];
    const int32_t m = mate[i];
    const int32_t lead = (m < 0 || m > i) ? i : m;
    comp[f] = id[lead];
  }
}

__global__ void k_iota(int64_t n, int32_t* a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (int32_t)i;
}

__global__ void k_member_fill(int64_t n, const int32_t* agg, int stride, int32_t* cnt,
                              int32_t* members, int* status) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t I = agg[i];
    const int slot = atomicAdd(&cnt[I], 1);
    if (slot < stride)
      members[(int64_t)I * stride + slot] = (int32_t)i;
    else
      atomicExch(status, AMG_ERR_DEVICE_CHECK);
  }
}

__global__ void k_member_sort(int64_t nc, int stride, const int32_t* cnt, int32_t* members) {
  for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < nc;
       I += (int64_t)gridDim.x * blockDim.x) {
    int32_t* m = members + I * stride;
    const int c = min(cnt[I], stride);
    for (int a = 1; a < c; ++a) {
      int32_t v = m[a];
      int b = a - 1;
      while (b >= 0 && m[b] > v) {
        m[b + 1] = m[b];
        --b;
      }
      m[b + 1] = v;
    }
    for (int a = c; a < stride; ++a) m[a] = -1;
  }
}

static int build_members(Arena& ar, int64_t n, const int32_t* agg, int64_t nc, int stride,
                         int32_t* members, int* dev_status, int num_sms, cudaStream_t s) {
  int32_t* cnt = nullptr;
  AMG_TRY(ar.alloc_n(&cnt, nc));
  AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nc, s));
  k_member_fill<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(n, agg, stride, cnt, members,
                                                             dev_status);
  AMG_LAUNCH_CHECK();
  k_member_sort<<<grid_for(nc, 256, num_sms, 8), 256, 0, s>>>(nc, stride, cnt, members);
  AMG_LAUNCH_CHECK();
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  ar.release(cnt);
  return AMG_OK;
}

// ------------------------------------------------------------------ Galerkin
// (A_c)_IJ = sum of a_ij over agg(i) = I, agg(j) = J, added left to right in
// ascending (min(i,j), max(i,j), [i > j]) order.  For each coarse row a team
// (one warp, or one block for long rows) stages the contributions of its
// member rows in shared memory, sorts them by (J, min, max, flip) with a
// bitonic network and adds each J-run sequentially.

constexpr int GAL_WARP_CAP = 512;   // contributions per warp-staged row
constexpr int GAL_WARPS = 4;        // warps per block in the warp kernel
constexpr int GAL_BLOCK_CAP = 8192; // contributions per block-staged row
constexpr int GAL_BLOCK_THREADS = 512;

__device__ __forceinline__ bool gless(uint64_t a1, uint64_t a2, uint64_t b1, uint64_t b2) {
  return a1 < b1 || (a1 == b1 && a2 < b2);
}

template <bool WARP>
__device__ __forceinline__ void team_sync() {
  if (WARP)
    __syncwarp();
  else
    __syncthreads();
}

template <bool WARP>
__device__ void bitonic_sort(uint64_t* k1, uint64_t* k2, double* v, int P, int tid, int tsz) {
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = tid; t < (P >> 1); t += tsz) {
        const int i = 2 * stride * (t / stride) + (t % stride);
        const int j = i + stride;
        const bool up = (i & size) == 0;
        const bool sw = up ? gless(k1[j], k2[j], k1[i], k2[i]) : gless(k1[i], k2[i], k1[j], k2[j]);
        if (sw) {
          uint64_t a = k1[i], b = k2[i];
          double c = v[i];
          k1[i] = k1[j];
          k2[i] = k2[j];
          v[i] = v[j];
          k1[j] = a;
          k2[j] = b;
          v[j] = c;
        }
      }
      team_sync<WARP>();
    }
  }
}

struct GalArgs {
  int64_t nc;
  int stride;
  const int32_t* members;
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
  const int32_t* agg;
  int64_t* cnt;           // count pass: distinct J per coarse row
  const int64_t* rowptr_c;  // fill pass
  int32_t* col_c;
  double* val_c;
  int32_t* ovf_list;      // rows staged by the block kernel
  int* ovf_count;
  int* status;
};

__device__ __forceinline__ int64_t gal_total(const GalArgs& g, int64_t I) {
  int64_t tot = 0;
  for (int s = 0; s < g.stride; ++s) {
    const int32_t m = g.members[I * g.stride + s];
    if (m < 0) break;
    tot += g.rowptr[m + 1] - g.rowptr[m];
  }
  return tot;
}

template <bool WARP>
__device__ void gal_stage(const GalArgs& g, int64_t I, uint64_t* k1, uint64_t* k2, double* v,
                          int total, int P, int tid, int tsz) {
  int pos = 0;
  for (int s = 0; s < g.stride; ++s) {
    const int32_t m = g.members[I * g.stride + s];
    if (m < 0) break;
    const int64_t beg = g.rowptr[m], end = g.rowptr[m + 1];
    for (int64_t e = beg + tid; e < end; e += tsz) {
      const int32_t j = g.col[e];
      const uint32_t J = (uint32_t)g.agg[j];
      const uint32_t lo = (uint32_t)min(m, j), hi = (uint32_t)max(m, j);
      const int p = pos + (int)(e - beg);
      k1[p] = ((uint64_t)J << 32) | lo;
      k2[p] = ((uint64_t)hi << 1) | (uint64_t)(m > j ? 1 : 0);
      v[p] = g.val[e];
    }
    pos += (int)(end - beg);
  }
  for (int p = total + tid; p < P; p += tsz) {
    k1[p] = ~0ull;
    k2[p] = ~0ull;
    v[p] = 0.0;
  }
  team_sync<WARP>();
}

__device__ __forceinline__ int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

template <bool FILL>
__global__ void __launch_bounds__(GAL_WARPS * 32) k_galerkin_warp(GalArgs g) {
  extern __shared__ unsigned char smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint64_t* k1 = (uint64_t*)smem + (size_t)wib * GAL_WARP_CAP;
  uint64_t* k2 = (uint64_t*)smem + (size_t)(GAL_WARPS + wib) * GAL_WARP_CAP;
  double* v = (double*)((uint64_t*)smem + (size_t)2 * GAL_WARPS * GAL_WARP_CAP) +
              (size_t)wib * GAL_WARP_CAP;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < g.nc; I += nw) {
    const int64_t tot64 = gal_total(g, I);
    if (tot64 > GAL_WARP_CAP) {
      if (!FILL && lane == 0) {
        const int k = atomicAdd(g.ovf_count, 1);
        g.ovf_list[k] = (int32_t)I;
        g.cnt[I] = 0;
      }
      continue;
    }
    const int total = (int)tot64;
    const int P = next_pow2(total);
    gal_stage<true>(g, I, k1, k2, v, total, P, lane, 32);
    bitonic_sort<true>(k1, k2, v, P, lane, 32);
    int base = 0;
    const int64_t off = FILL ? g.rowptr_c[I] : 0;
    for (int c = 0; c < total; c += 32) {
      const int p = c + lane;
      const bool st = p < total && (p == 0 || (k1[p] >> 32) != (k1[p - 1] >> 32));
      const unsigned msk = __ballot_sync(0xffffffffu, st);
      if (FILL && st) {
        const int rank = base + __popc(msk & ((1u << lane) - 1u));
        const uint64_t J = k1[p] >> 32;
        double s = v[p];
        for (int q = p + 1; q < total && (k1[q] >> 32) == J; ++q) s = __dadd_rn(s, v[q]);
        g.col_c[off + rank] = (int32_t)J;
        g.val_c[off + rank] = s;
      }
      base += __popc(msk);
    }
    if (!FILL && lane == 0) g.cnt[I] = base;
    __syncwarp();
  }
}

// Long rows: one block per listed row, staging up to GAL_BLOCK_CAP entries.
template <bool FILL>
__global__ void __launch_bounds__(GAL_BLOCK_THREADS) k_galerkin_block(GalArgs g, int nrows) {
  extern __shared__ unsigned char smem[];
  uint64_t* k1 = (uint64_t*)smem;
  uint64_t* k2 = k1 + GAL_BLOCK_CAP;
  double* v = (double*)(k2 + GAL_BLOCK_CAP);
  for (int r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int64_t I = g.ovf_list[r];
    const int64_t tot64 = gal_total(g, I);
    if (tot64 > GAL_BLOCK_CAP) {
      if (threadIdx.x == 0) {
        atomicExch(g.status, AMG_ERR_UNSUPPORTED);
        if (!FILL) g.cnt[I] = 0;
      }
      continue;
    }
    const int total = (int)tot64;
    const int P = next_pow2(total);
    gal_stage<false>(g, I, k1, k2, v, total, P, threadIdx.x, blockDim.x);
    bitonic_sort<false>(k1, k2, v, P, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) {  // rare: sequential run-length pass
      const int64_t off = FILL ? g.rowptr_c[I] : 0;
      int rank = 0;
      int p = 0;
      while (p < total) {
        const uint64_t J = k1[p] >> 32;
        double s = v[p];
        int q = p + 1;
        for (; q < total && (k1[q] >> 32) == J; ++q) s = __dadd_rn(s, v[q]);
        if (FILL) {
          g.col_c[off + rank] = (int32_t)J;
          g.val_c[off + rank] = s;
        }
        ++rank;
        p = q;
      }
      if (!FILL) g.cnt[I] = rank;
    }
    __syncthreads();
  }
}

// Coarse CSR of P^T A P for aggregates `agg` with member lists `members`.
static int galerkin(Arena& ar, int64_t n, const int64_t* rowptr, const int32_t* col,
                    const double* val, const int32_t* agg, const int32_t* members, int stride,
                    int64_t nc, int64_t** rp_c, int32_t** col_c, double** val_c, int64_t* nnz_c,
                    int* dev_status, int num_sms, cudaStream_t s) {
  (void)n;
  GalArgs g;
  g.nc = nc;
  g.stride = stride;
  g.members = members;
  g.rowptr = rowptr;
  g.col = col;
  g.val = val;
  g.agg = agg;
  g.status = dev_status;
  AMG_TRY(ar.alloc_n(&g.cnt, nc + 1));
  AMG_CUDA_TRY(cudaMemsetAsync(g.cnt, 0, sizeof(int64_t) * (nc + 1), s));
  AMG_TRY(ar.alloc_n(&g.ovf_list, nc));
  AMG_TRY(ar.alloc_n(&g.ovf_count, 1));
  AMG_CUDA_TRY(cudaMemsetAsync(g.ovf_count, 0, sizeof(int), s));
  const size_t wsm = (size_t)GAL_WARPS * GAL_WARP_CAP * 24;
  const size_t bsm = (size_t)GAL_BLOCK_CAP * 24;
  AMG_CUDA_TRY(cudaFuncSetAttribute(k_galerkin_block<false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
  AMG_CUDA_TRY(cudaFuncSetAttribute(k_galerkin_block<true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
  const int wgrid = grid_for(nc * 32, GAL_WARPS * 32, num_sms, 16);
  g.rowptr_c = nullptr;
  g.col_c = nullptr;
  g.val_c = nullptr;
  k_galerkin_warp<false><<<wgrid, GAL_WARPS * 32, wsm, s>>>(g);
  AMG_LAUNCH_CHECK();
  int novf = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&novf, g.ovf_count, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  if (novf > 0) {
    k_galerkin_block<false><<<std::min(novf, num_sms * 2), GAL_BLOCK_THREADS, bsm, s>>>(g, novf);
    AMG_LAUNCH_CHECK();
  }
  AMG_TRY(ar.alloc_n(rp_c, nc + 1));
  int64_t total = 0;
  AMG_TRY(scan_exclusive_i64(ar, g.cnt, *rp_c, nc + 1, &total, s));  // cnt[nc] unused -> last
  *nnz_c = total;
  AMG_TRY(ar.alloc_n(col_c, total));
  AMG_TRY(ar.alloc_n(val_c, total));
  g.rowptr_c = *rp_c;
  g.col_c = *col_c;
  g.val_c = *val_c;
  k_galerkin_warp<true><<<wgrid, GAL_WARPS * 32, wsm, s>>>(g);
  AMG_LAUNCH_CHECK();
  if (novf > 0) {
    k_galerkin_block<true><<<std::min(novf, num_sms * 2), GAL_BLOCK_THREADS, bsm, s>>>(g, novf);
    AMG_LAUNCH_CHECK();
  }
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  ar.release(g.cnt);
  ar.release(g.ovf_list);
  ar.release(g.ovf_count);
  return AMG_OK;
}

// ------------------------------------------------------------------ coarse Cholesky

// The coarsest matrix is block diagonal: one block (system) per CUDA block.
// Block b covers rows [brow[b], brow[b+1]); its dense row-major copy, L^-1
// and L^-T start at bmat[b].
__global__ void k_dense_blocks(const int64_t* rowptr, const int32_t* col, const double* val,
                               const int64_t* brow, const int64_t* bmat, double* dense,
                               int* status) {
  const int64_t r0 = brow[blockIdx.x], n = brow[blockIdx.x + 1] - r0;
  double* a = dense + bmat[blockIdx.x];
  for (int64_t t = threadIdx.x; t < n * n; t += blockDim.x) a[t] = 0.0;
  __syncthreads();
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = rowptr[r0 + i] + threadIdx.x; e < rowptr[r0 + i + 1]; e += blockDim.x) {
      const int64_t j = col[e] - r0;
      if (j >= 0 && j < n)
        a[i * n + j] = val[e];
      else
        atomicExch(status, AMG_ERR_DEVICE_CHECK);  // an entry coupling two blocks
    }
}

// Right-looking Cholesky of each block; the dense copy becomes L in its lower
// triangle.  Then L^-1 (one column per thread) and its transpose.
__global__ void k_cholesky(const int64_t* brow, const int64_t* bmat, double* dense,
                           double* Linv_all, double* LinvT_all, int* status) {
  const int n = (int)(brow[blockIdx.x + 1] - brow[blockIdx.x]);
  double* a = dense + bmat[blockIdx.x];
  double* Linv = Linv_all + bmat[blockIdx.x];
  double* LinvT = LinvT_all + bmat[blockIdx.x];
  __shared__ int ok;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double piv = a[(int64_t)k * n + k];
      ok = piv > 0.0;
      if (ok) a[(int64_t)k * n + k] = sqrt(piv);
    }
    __syncthreads();
    if (!ok) {
      if (threadIdx.x == 0) atomicExch(status, AMG_ERR_NOT_SPD);
      return;
    }
    const double lkk = a[(int64_t)k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x)
      a[(int64_t)i * n + k] = __ddiv_rn(a[(int64_t)i * n + k], lkk);
    __syncthreads();
    const int m = n - k - 1;
    for (int64_t idx = threadIdx.x; idx < (int64_t)m * m; idx += blockDim.x) {
      const int ii = (int)(idx / m), jj = (int)(idx % m);
      if (jj <= ii) {
        const int i = k + 1 + ii, j = k + 1 + jj;
        a[(int64_t)i * n + j] = __dsub_rn(a[(int64_t)i * n + j],
                                          __dmul_rn(a[(int64_t)i * n + k], a[(int64_t)j * n + k]));
      }
    }
    __syncthreads();
  }
  // column c of L^-1 by forward substitution on e_c
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    for (int i = 0; i < c; ++i) Linv[(int64_t)i * n + c] = 0.0;
    for (int i = c; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k)
        s = __dsub_rn(s, __dmul_rn(a[(int64_t)i * n + k], Linv[(int64_t)k * n + c]));
      Linv[(int64_t)i * n + c] = __ddiv_rn(s, a[(int64_t)i * n + i]);
    }
  }
  __syncthreads();
  for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    LinvT[(int64_t)j * n + i] = Linv[idx];
  }
}

// Blocked right-looking Cholesky for large coarsest blocks (several CUDA
// blocks per step).  Every entry receives the same rank-1 updates, in the
// same column order and with the same explicitly rounded operations, as in
// the one-block kernel above, so both produce the same factor bit for bit.
constexpr int CHOL_NB = 32;

// Factor the diagonal tile [kb, kb+nb) in place (one CUDA block).
__global__ void k_chol_diag(double* a, int64_t n, int64_t kb, int nb, int* status) {
  __shared__ int ok;
  for (int k = 0; k < nb; ++k) {
    const int64_t kk = kb + k;
    if (threadIdx.x == 0) {
      const double piv = a[kk * n + kk];
      ok = piv > 0.0;
      if (ok) a[kk * n + kk] = sqrt(piv);
    }
    __syncthreads();
    if (!ok) {
      if (threadIdx.x == 0) atomicExch(status, AMG_ERR_NOT_SPD);
      return;
    }
    const double lkk = a[kk * n + kk];
    for (int i = k + 1 + threadIdx.x; i < nb; i += blockDim.x)
      a[(kb + i) * n + kk] = __ddiv_rn(a[(kb + i) * n + kk], lkk);
    __syncthreads();
    const int m = nb - k - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int ii = idx / m, jj = idx % m;
      if (jj <= ii) {
        const int64_t i = kb + k + 1 + ii, j = kb + k + 1 + jj;
        a[i * n + j] = __dsub_rn(a[i * n + j], __dmul_rn(a[i * n + kk], a[j * n + kk]));
      }
    }
    __syncthreads();
  }
}

// Panel below the tile: row i >= kb+nb, columns k = kb..kb+nb-1 in order.
__global__ void k_chol_panel(double* a, int64_t n, int64_t kb, int nb) {
  for (int64_t i = kb + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < nb; ++k) {
      const int64_t kk = kb + k;
      double v = a[i * n + kk];
      for (int q = 0; q < k; ++q)
        v = __dsub_rn(v, __dmul_rn(a[i * n + kb + q], a[kk * n + kb + q]));
      a[i * n + kk] = __ddiv_rn(v, a[kk * n + kk]);
    }
  }
}

// Trailing update: a_ij -= l_ik l_jk for k = kb..kb+nb-1 in order, j <= i.
__global__ void k_chol_update(double* a, int64_t n, int64_t kb, int nb) {
  const int64_t t0 = kb + nb, m = n - t0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < m * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ii = idx / m, jj = idx % m;
    if (jj > ii) continue;
    const int64_t i = t0 + ii, j = t0 + jj;
    double v = a[i * n + j];
    for (int k = 0; k < nb; ++k)
      v = __dsub_rn(v, __dmul_rn(a[i * n + kb + k], a[j * n + kb + k]));
    a[i * n + j] = v;
  }
}

// Column c of L^-1 per thread (forward substitution on e_c), then L^-T.
__global__ void k_tri_inverse(const double* a, int64_t n, double* Linv) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t i = 0; i < c; ++i) Linv[i * n + c] = 0.0;
    for (int64_t i = c; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int64_t k = c; k < i; ++k) s = __dsub_rn(s, __dmul_rn(a[i * n + k], Linv[k * n + c]));
      Linv[i * n + c] = __ddiv_rn(s, a[i * n + i]);
    }
  }
}

__global__ void k_transpose(const double* in, int64_t n, double* out) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
       idx += (int64_t)gridDim.x * blockDim.x)
    out[(idx % n) * n + idx / n] = in[idx];
}

static int chol_blocked(double* a, int64_t n, double* Linv, double* LinvT, int* status,
                        int num_sms, cudaStream_t s) {
  for (int64_t kb = 0; kb < n; kb += CHOL_NB) {
    const int nb = (int)std::min<int64_t>(CHOL_NB, n - kb);
    k_chol_diag<<<1, 256, 0, s>>>(a, n, kb, nb, status);
    AMG_LAUNCH_CHECK();
    if (kb + nb < n) {
      k_chol_panel<<<grid_for(n - kb - nb, 128, num_sms, 4), 128, 0, s>>>(a, n, kb, nb);
      AMG_LAUNCH_CHECK();
      const int64_t m = n - kb - nb;
      k_chol_update<<<grid_for(m * m, 256, num_sms, 8), 256, 0, s>>>(a, n, kb, nb);
      AMG_LAUNCH_CHECK();
    }
  }
  k_tri_inverse<<<grid_for(n, 64, num_sms, 8), 64, 0, s>>>(a, n, Linv);
  AMG_LAUNCH_CHECK();
  k_transpose<<<grid_for(n * n, 256, num_sms, 8), 256, 0, s>>>(Linv, n, LinvT);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// ------------------------------------------------------------------ V-cycle operators
// AP = A P: row i holds every aggregate J among agg(col(i, :)) once, in order
// of first appearance, with the sum of its entries taken in column order.

__device__ __forceinline__ bool seen_before(const int64_t* rowptr_i, const int32_t* col,
                                            const int32_t* agg, int64_t e, int32_t J) {
  for (int64_t f = *rowptr_i; f < e; ++f)
    if (agg[col[f]] == J) return true;
  return false;
}

__global__ void k_ap_count(int64_t n, const int64_t* rowptr, const int32_t* col,
                           const int32_t* agg, int64_t* cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = 0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (!seen_before(rowptr + i, col, agg, e, agg[col[e]])) ++c;
    cnt[i] = c;
  }
}

__global__ void k_ap_fill(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                          const int32_t* agg, const int64_t* rp_ap, int32_t* col_ap,
                          double* val_ap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t pos = rp_ap[i];
    const int64_t end = rowptr[i + 1];
    for (int64_t e = rowptr[i]; e < end; ++e) {
      const int32_t J = agg[col[e]];
      if (seen_before(rowptr + i, col, agg, e, J)) continue;
      double s = val[e];
      for (int64_t f = e + 1; f < end; ++f)
        if (agg[col[f]] == J) s = __dadd_rn(s, val[f]);
      col_ap[pos] = J;
      val_ap[pos] = s;
      ++pos;
    }
  }
}

// Ah values: a_ij * s_j on A's sliced-ELL slots (padding stays 0).  Each
// thread takes SC_U slots a grid stride apart per step and issues all their
// loads, then all their gathers, before any product, so that SC_U times the
// bytes of a one-slot loop are in flight.
constexpr int SC_U = 4;
__global__ void k_scale_cols(int64_t m, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ s,
                             double* __restrict__ out64, float* __restrict__ out32,
                             __nv_bfloat16* __restrict__ out16) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e0 < m;
       e0 += SC_U * stride) {
    int32_t c[SC_U];
    double a[SC_U], sj[SC_U];
#pragma unroll
    for (int u = 0; u < SC_U; ++u) {
      const int64_t e = e0 + u * stride;
      c[u] = e < m ? ld_stream(col + e) : 0;
      a[u] = e < m ? ld_stream(val + e) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < SC_U; ++u) sj[u] = e0 + u * stride < m ? __ldg(s + c[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < SC_U; ++u) {
      const int64_t e = e0 + u * stride;
      if (e < m) {
        const double v = __dmul_rn(a[u], sj[u]);
        out64[e] = v;
        if (out32) out32[e] = (float)v;
        if (out16) out16[e] = __float2bfloat16_rn((float)v);
      }
    }
  }
}

static int build_ah(Arena& ar, Level& L, int num_sms, cudaStream_t s) {
  const int64_t m = L.A.nnz_pad;
  if (!L.ah64) AMG_TRY(ar.alloc_n(&L.ah64, m));
  if (L.vstore == VAL_F32 && !L.ah32) AMG_TRY(ar.alloc_n(&L.ah32, m));
  if (L.vstore == VAL_BF16 && !L.ah16) AMG_TRY(ar.alloc_n(&L.ah16, m));
  int occ = 0;  // a grid of the CTAs that fit at once (no partial second wave)
  AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_scale_cols, 256, 0));
  k_scale_cols<<<grid_for((m + SC_U - 1) / SC_U, 256, num_sms, std::max(occ, 1)), 256, 0, s>>>(
      m, L.A.col, L.A.v64, L.s64, L.ah64, L.ah32, L.ah16);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

static int build_ap(Arena& ar, Level& L, const int64_t* rp, const int32_t* ci, const double* va,
                    bool compress, int num_sms, cudaStream_t s) {
  const int64_t n = L.n;
  int64_t* cnt = nullptr;
  int64_t* rp_ap = nullptr;
  AMG_TRY(ar.alloc_n(&cnt, n + 1));
  AMG_TRY(ar.alloc_n(&rp_ap, n + 1));
  AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (n + 1), s));
  const int g = grid_for(n, 256, num_sms, 8);
  k_ap_count<<<g, 256, 0, s>>>(n, rp, ci, L.agg, cnt);
  AMG_LAUNCH_CHECK();
  int64_t total = 0;
  AMG_TRY(scan_exclusive_i64(ar, cnt, rp_ap, n + 1, &total, s));
  int32_t* ci_ap = nullptr;
  double* va_ap = nullptr;
  AMG_TRY(ar.alloc_n(&ci_ap, total));
  AMG_TRY(ar.alloc_n(&va_ap, total));
  k_ap_fill<<<g, 256, 0, s>>>(n, rp, ci, va, L.agg, rp_ap, ci_ap, va_ap);
  AMG_LAUNCH_CHECK();
  L.ap_nnz = total;
  AMG_TRY(sell_from_csr(ar, n, L.nc, rp_ap, ci_ap, va_ap, L.A.C, L.A.tpr, L.AP, s,
                        L.sys_off.empty() ? nullptr : &L.sys_off, compress));
  if (L.vstore != VAL_F64) AMG_TRY(sell_make_copies(ar, L.AP, L.vstore, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  ar.release(cnt);
  ar.release(rp_ap);
  ar.release(ci_ap);
  ar.release(va_ap);
  return AMG_OK;
}

// Coarse matrix with the smoothed prolongator (Sec. 2.3, SMATCH): A P_hat
// (k_ap_*: per row, each aggregate's sum in stored order), P = P_hat -
// w D^-1 (A P_hat) in place, R = P^T, Q = A P and A_c = R Q, every sum in
// ascending inner index.  P, R and Q stay on the level until setup has built
// the V-cycle operators from them.
static int smoothed_galerkin(Arena& ar, Level& L, int64_t n, const int64_t* rp,
                             const int32_t* ci, const double* va, Level& next, double pfilter,
                             int* dev_status, int num_sms, cudaStream_t s) {
  // the matrix P is smoothed with: A, or A_F (option prolongator_filter)
  int64_t* f_rp = nullptr;
  int32_t* f_ci = nullptr;
  double* f_va = nullptr;
  const int64_t* srp = rp;
  const int32_t* sci = ci;
  const double* sva = va;
  if (pfilter > 0.0) {
    double* diag = nullptr;
    AMG_TRY(ar.alloc_n(&diag, n));
    k_l1_diag<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(n, rp, ci, va, nullptr, diag);
    AMG_LAUNCH_CHECK();
    AMG_TRY(filter_matrix(ar, n, rp, ci, va, diag, pfilter, &f_rp, &f_ci, &f_va, num_sms, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    ar.release(diag);
    srp = f_rp;
    sci = f_ci;
    sva = f_va;
  }
  int64_t* cnt = nullptr;
  AMG_TRY(ar.alloc_n(&cnt, n + 1));
  AMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int64_t) * (n + 1), s));
  const int g = grid_for(n, 256, num_sms, 8);
  k_ap_count<<<g, 256, 0, s>>>(n, srp, sci, L.agg, cnt);
  AMG_LAUNCH_CHECK();
  AMG_TRY(ar.alloc_n(&L.p_rp, n + 1));
  AMG_TRY(scan_exclusive_i64(ar, cnt, L.p_rp, n + 1, &L.p_nnz, s));
  ar.release(cnt);
  AMG_TRY(ar.alloc_n(&L.p_ci, L.p_nnz));
  AMG_TRY(ar.alloc_n(&L.p_v, L.p_nnz));
  k_ap_fill<<<g, 256, 0, s>>>(n, srp, sci, sva, L.agg, L.p_rp, L.p_ci, L.p_v);
  AMG_LAUNCH_CHECK();
  // D and w come from A itself; only the product A_F P_hat is filtered
  AMG_TRY(smoothed_prolongator(ar, n, rp, ci, va, L.agg, L.p_rp, L.p_ci, L.p_v, &L.wp, num_sms,
                               s));
  if (pfilter > 0.0) {
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    for (void* p : {(void*)f_rp, (void*)f_ci, (void*)f_va}) ar.release(p);
  }
  AMG_TRY(transpose_csr(ar, n, L.nc, L.p_rp, L.p_ci, L.p_v, L.p_nnz, &L.t_rp, &L.t_ci, &L.t_v,
                        num_sms, s));
  AMG_TRY(spgemm(ar, n, rp, ci, va, L.p_rp, L.p_ci, L.p_v, &L.q_rp, &L.q_ci, &L.q_v, &L.q_nnz,
                 dev_status, num_sms, s));
  AMG_TRY(spgemm(ar, L.nc, L.t_rp, L.t_ci, L.t_v, L.q_rp, L.q_ci, L.q_v, &next.rowptr, &next.col,
                 &next.val, &next.nnz, dev_status, num_sms, s));
  return AMG_OK;
}

// Threads per row when the options fix none: one (32 rows a slice) for
// ordinary rows; rows of 64 entries or more (coarse levels of smoothed
// hierarchies reach hundreds) get a power of two from 4 up to a whole warp,
// about one thread per 16 entries.  FP64 operators larger than the L2 get
// one thread per 32: each halving of the threads per row removes a level of
// the cross-lane FP64 reduction (shuffle and add chain; at 16 threads a
// 140-entry row spent 64 additions on it, with the FP64 pipe 76% busy) and
// gives each lane more independent loads; smaller operators stay in L2, are
// latency bound, and want the threads.
constexpr double L2_OPERATOR_BYTES = 126.0 * 1024 * 1024;

static int auto_tpr(int64_t rows, int64_t nnz, bool f64) {
  const double m = (double)nnz / (double)std::max<int64_t>(rows, 1);
  if (m < 64.0) return 1;
  const double per = f64 && 12.0 * (double)nnz > L2_OPERATOR_BYTES ? 32.0 : 16.0;
  int t = 4;
  while (t < 32 && per * t < m) t <<= 1;
  return t;
}

// Sliced-ELL copies of A P, P (both with A's slices and plain column
// indices, so one kernel walks both with the same layout code) and R = P^T
// of a smoothed level; R's rows (the fine rows around an aggregate) are
// long, so it gets its own threads per row (at least 4 once they average 16
// entries).
static int build_smoothed_ops(Arena& ar, Level& L, bool compress, cudaStream_t s) {
  L.ap_nnz = L.q_nnz;
  AMG_TRY(sell_from_csr(ar, L.n, L.nc, L.q_rp, L.q_ci, L.q_v, L.A.C, L.A.tpr, L.AP, s, nullptr,
                        false));
  AMG_TRY(sell_from_csr(ar, L.n, L.nc, L.p_rp, L.p_ci, L.p_v, L.A.C, L.A.tpr, L.P, s, nullptr,
                        false));
  const int rt = std::max(auto_tpr(L.nc, L.p_nnz, L.vstore == VAL_F64),
                          L.p_nnz >= 16 * L.nc ? 4 : 1);
  AMG_TRY(sell_from_csr(ar, L.nc, L.n, L.t_rp, L.t_ci, L.t_v, 32 / rt, rt, L.R, s, nullptr,
                        compress));
  if (L.vstore != VAL_F64)
    for (Sell* M : {&L.AP, &L.P, &L.R}) AMG_TRY(sell_make_copies(ar, *M, L.vstore, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  for (void* p : {(void*)L.t_rp, (void*)L.t_ci, (void*)L.t_v, (void*)L.q_rp, (void*)L.q_ci,
                  (void*)L.q_v})
    ar.release(p);
  L.t_rp = L.q_rp = nullptr;
  L.t_ci = L.q_ci = nullptr;
  L.t_v = L.q_v = nullptr;
  return AMG_OK;
}

// ------------------------------------------------------------------ autotuner
// Slice height C and threads per row per level, chosen by timing the level's
// smoother kernels (and the level-0 SpMV) in every candidate layout; choices
// are remembered for the process, keyed by (rows, 10 x entries per row, value
// type, batched, compressed columns).

struct TuneKey {
  int64_t n;
  int nnz10;
  int vstore;
  bool batched;
  bool compress;
  bool operator<(const TuneKey& o) const {
    if (n != o.n) return n < o.n;
    if (nnz10 != o.nnz10) return nnz10 < o.nnz10;
    if (vstore != o.vstore) return vstore < o.vstore;
    if (batched != o.batched) return batched < o.batched;
    return compress < o.compress;
  }
};

struct Layout {
  int C, tpr;
};

static std::mutex g_tune_mu;
static std::map<TuneKey, Layout> g_tune;

static bool tune_lookup(const TuneKey& k, Layout* lay) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *lay = it->second;
  return true;
}

static void tune_store(const TuneKey& k, Layout lay) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[k] = lay;
}

// Candidate layouts of a level: threads per row 1, 2, 4, 8 (and 16, 32 when
// rows average 64 entries or more) with slice height 32 / tpr, and, unless
// the slices must follow the warps (batched systems), heights 8, 16, 32, 64.
static std::vector<Layout> tune_candidates(bool wide, bool batched) {
  std::vector<Layout> c;
  for (int tpr = 1; tpr <= (wide ? 32 : 8); tpr <<= 1) {
    c.push_back({32 / tpr, tpr});
    if (batched) continue;
    for (int C : {8, 16, 32, 64})
      if (C != 32 / tpr) c.push_back({C, tpr});
  }
  return c;
}

static void release_sell(Arena& ar, Sell& A) {
  for (void* p : {(void*)A.sliceptr, (void*)A.col, (void*)A.v64, (void*)A.v32, (void*)A.v16,
                  (void*)A.row0, (void*)A.sys, (void*)A.d16, (void*)A.kbase})
    ar.release(p);
  A = Sell();
}

static void release_level_ops(Arena& ar, Level& L) {
  release_sell(ar, L.A);
  release_sell(ar, L.AP);
  release_sell(ar, L.P);
  release_sell(ar, L.R);
  ar.release(L.ah64);
  ar.release(L.ah32);
  ar.release(L.ah16);
  L.ah64 = nullptr;
  L.ah32 = nullptr;
  L.ah16 = nullptr;
  L.ap_nnz = 0;
}

// ------------------------------------------------------------------ driver

int set_level0_weights(amg_handle* H, const float* omega, cudaStream_t s) {
  Level& L = H->L[0];
  k_smoother_scale<<<grid_for(L.n, 256, H->num_sms, 8), 256, 0, s>>>(L.n, L.dinv, omega, L.s64,
                                                                     L.s32);
  AMG_LAUNCH_CHECK();
  if (L.ah64) AMG_TRY(build_ah(H->arena, L, H->num_sms, s));
  return AMG_OK;
}

// Largest system of a batched level (each keeps the coarsest level it would
// get alone); the whole level otherwise.
static int64_t largest_block(const Level& L, int64_t n) {
  if (L.sys_off.size() < 2) return n;
  int64_t m = 0;
  for (size_t k = 0; k + 1 < L.sys_off.size(); ++k)
    m = std::max(m, L.sys_off[k + 1] - L.sys_off[k]);
  return m;
}

static int read_status(amg_handle* H, cudaStream_t s) {
  int h = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&h, H->dev_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  return h;
}

int setup_hierarchy(amg_handle* H, const amg_csr* A, cudaStream_t s, const amg_handle* like) {
  const amg_options& o = H->opt;
  Arena& ar = H->arena;
  const int sms = H->num_sms;
  const bool f32 = o.precision == AMG_PREC_F32;
  H->L.clear();
  H->L.emplace_back();
  H->L[0].n = A->n;
  H->L[0].nnz = A->nnz;
  if (H->batched) H->L[0].sys_off = H->sys_off0;
  const int stride = 1 << o.sweeps;
  for (int l = 0;; ++l) {
    const int64_t n = H->L[l].n;
    const int64_t* rp = l == 0 ? A->rowptr : H->L[l].rowptr;
    const int32_t* ci = l == 0 ? A->col : H->L[l].col;
    const double* va = l == 0 ? A->val : H->L[l].val;
    double* diag = nullptr;
    AMG_TRY(ar.alloc_n(&H->L[l].d, n));
    AMG_TRY(ar.alloc_n(&H->L[l].dinv, n));
    AMG_TRY(ar.alloc_n(&H->L[l].s64, n));
    if (f32) AMG_TRY(ar.alloc_n(&H->L[l].s32, n));
    AMG_TRY(ar.alloc_n(&diag, n));
    const int g1 = grid_for(n, 256, sms, 8);
    k_l1_diag<<<g1, 256, 0, s>>>(n, rp, ci, va, H->L[l].d, diag);
    AMG_LAUNCH_CHECK();
    k_recip<<<g1, 256, 0, s>>>(n, H->L[l].d, H->L[l].dinv);
    AMG_LAUNCH_CHECK();
    k_smoother_scale<<<g1, 256, 0, s>>>(n, H->L[l].dinv, nullptr, H->L[l].s64, H->L[l].s32);
    AMG_LAUNCH_CHECK();
    if (like) {  // new values on an assembled hierarchy: its aggregates, no matching
      ar.release(diag);
      if (l + 1 >= (int)like->L.size()) break;
      Level& L = H->L[l];
      const Level& K = like->L[l];
      L.nc = K.nc;
      L.stride = K.stride;
      AMG_TRY(ar.alloc_n(&L.agg, n));
      AMG_TRY(ar.alloc_n(&L.members, L.nc * L.stride));
      AMG_CUDA_TRY(cudaMemcpyAsync(L.agg, K.agg, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice,
                                   s));
      AMG_CUDA_TRY(cudaMemcpyAsync(L.members, K.members, sizeof(int32_t) * L.nc * L.stride,
                                   cudaMemcpyDeviceToDevice, s));
      Level next;
      next.n = L.nc;
      if (o.smooth_prolongator)
        AMG_TRY(smoothed_galerkin(ar, L, n, rp, ci, va, next, o.prolongator_filter,
                                  H->dev_status, sms, s));
      else
        AMG_TRY(galerkin(ar, n, rp, ci, va, L.agg, L.members, L.stride, L.nc, &next.rowptr,
                         &next.col, &next.val, &next.nnz, H->dev_status, sms, s));
      const int st = read_status(H, s);
      if (st < 0) return st;
      H->L.push_back(next);
      continue;
    }
    if (largest_block(H->L[l], n) <= o.max_coarse || l + 1 >= o.max_levels) {
      ar.release(diag);
      break;
    }
    // k matching sweeps; sweep s+1 matches the Galerkin matrix of the
    // composite map after sweep s (aggregates <= 2^k).
    int32_t* comp = nullptr;
    AMG_TRY(ar.alloc_n(&comp, n));
    k_iota<<<g1, 256, 0, s>>>(n, comp);
    AMG_LAUNCH_CHECK();
    int64_t cn = n, nc = n;
    const int64_t* crp = rp;
    const int32_t* cci = ci;
    const double* cva = va;
    double* cdiag = diag;
    int64_t* t_rp = nullptr;
    int32_t* t_ci = nullptr;
    double* t_va = nullptr;
    int lstride = stride;  // member-table width of this level
    if (o.aggregation == 1)
      AMG_TRY(vbm_aggregate(ar, n, rp, ci, va, diag, o.vbm_theta, comp, &nc, &lstride, sms, s));
    for (int sw = 0; sw < o.sweeps && o.aggregation == 0; ++sw) {
      int32_t *mate = nullptr, *flag = nullptr, *id = nullptr;
      AMG_TRY(ar.alloc_n(&mate, cn));
      AMG_TRY(match_rounds(ar, cn, crp, cci, cva, cdiag, mate, nullptr, sms, s));
      AMG_TRY(ar.alloc_n(&flag, cn));
      AMG_TRY(ar.alloc_n(&id, cn));
      const int gc = grid_for(cn, 256, sms, 8);
      k_leader_flags<<<gc, 256, 0, s>>>(cn, mate, flag);
      AMG_LAUNCH_CHECK();
      AMG_TRY(scan_exclusive_i32(ar, flag, id, cn, &nc, s));
      k_assign_compose<<<g1, 256, 0, s>>>(n, cn, mate, id, comp);
      AMG_LAUNCH_CHECK();
      AMG_CUDA_TRY(cudaStreamSynchronize(s));
      ar.release(mate);
      ar.release(flag);
      ar.release(id);
      if (sw + 1 < o.sweeps) {
        const int st = 1 << (sw + 1);
        int32_t* mem = nullptr;
        AMG_TRY(ar.alloc_n(&mem, nc * st));
        AMG_TRY(build_members(ar, n, comp, nc, st, mem, H->dev_status, sms, s));
        int64_t* n_rp = nullptr;
        int32_t* n_ci = nullptr;
        double* n_va = nullptr;
        int64_t n_nnz = 0;
        AMG_TRY(galerkin(ar, n, rp, ci, va, comp, mem, st, nc, &n_rp, &n_ci, &n_va, &n_nnz,
                         H->dev_status, sms, s));
        ar.release(mem);
        ar.release(t_rp);
        ar.release(t_ci);
        ar.release(t_va);
        t_rp = n_rp;
        t_ci = n_ci;
        t_va = n_va;
        if (cdiag != diag) ar.release(cdiag);
        AMG_TRY(ar.alloc_n(&cdiag, nc));
        k_l1_diag<<<grid_for(nc, 256, sms, 8), 256, 0, s>>>(nc, t_rp, t_ci, t_va, nullptr, cdiag);
        AMG_LAUNCH_CHECK();
        crp = t_rp;
        cci = t_ci;
        cva = t_va;
        cn = nc;
      }
    }
    ar.release(t_rp);
    ar.release(t_ci);
    ar.release(t_va);
    if (cdiag != diag) ar.release(cdiag);
    ar.release(diag);
    int st = read_status(H, s);
    if (st < 0) return st;
    if ((double)nc > o.stall_ratio * (double)n) {
      ar.release(comp);
      break;
    }
    Level& L = H->L[l];
    L.agg = comp;
    L.nc = nc;
    L.stride = lstride;
    AMG_TRY(ar.alloc_n(&L.members, nc * lstride));
    AMG_TRY(build_members(ar, n, L.agg, nc, lstride, L.members, H->dev_status, sms, s));
    Level next;
    next.n = nc;
    if (H->batched) {  // aggregates never span systems: system k starts at agg(first row)
      next.sys_off.assign(H->nsys + 1, nc);
      for (int k = 0; k < H->nsys; ++k) {
        int32_t a = 0;
        AMG_CUDA_TRY(cudaMemcpyAsync(&a, L.agg + L.sys_off[k], sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s));
        AMG_CUDA_TRY(cudaStreamSynchronize(s));
        next.sys_off[k] = a;
      }
    }
    if (o.smooth_prolongator)
      AMG_TRY(smoothed_galerkin(ar, L, n, rp, ci, va, next, o.prolongator_filter,
                                  H->dev_status, sms, s));
    else
      AMG_TRY(galerkin(ar, n, rp, ci, va, L.agg, L.members, lstride, nc, &next.rowptr,
                       &next.col, &next.val, &next.nnz, H->dev_status, sms, s));
    st = read_status(H, s);
    if (st < 0) return st;
    H->L.push_back(next);
  }
  // coarsest level: dense Cholesky and its inverse factor
  // (block diagonal for batched systems: one dense factor per system), or
  // the work vectors of the PCG coarsest solve
  Level& Lc = H->L.back();
  H->nco = Lc.n;
  if (o.coarse_solver == 1) {
    H->nblk = 1;
    H->cblk_row = {0, Lc.n};
    AMG_TRY(ar.alloc_n(&H->cpcg, 5 * Lc.n));
  } else {
    if (largest_block(Lc, Lc.n) > o.max_dense) return AMG_ERR_UNSUPPORTED;
    std::vector<int64_t> brow = Lc.sys_off.size() >= 2 ? Lc.sys_off
                                                        : std::vector<int64_t>{0, Lc.n};
    const int nb = (int)brow.size() - 1;
    std::vector<int64_t> bmat(nb + 1, 0);
    for (int b = 0; b < nb; ++b)
      bmat[b + 1] = bmat[b] + (brow[b + 1] - brow[b]) * (brow[b + 1] - brow[b]);
    H->nblk = nb;
    H->cblk_row = brow;
    const int64_t* rp = H->L.size() == 1 ? A->rowptr : Lc.rowptr;
    const int32_t* ci = H->L.size() == 1 ? A->col : Lc.col;
    const double* va = H->L.size() == 1 ? A->val : Lc.val;
    double* dense = nullptr;
    AMG_TRY(ar.alloc_n(&dense, bmat.back()));
    AMG_TRY(ar.alloc_n(&H->Linv, bmat.back()));
    AMG_TRY(ar.alloc_n(&H->LinvT, bmat.back()));
    AMG_TRY(ar.alloc_n(&H->d_brow, nb + 1));
    AMG_TRY(ar.alloc_n(&H->d_bmat, nb + 1));
    AMG_TRY(ar.alloc_n(&H->coarse_y, Lc.n));
    AMG_CUDA_TRY(cudaMemcpyAsync(H->d_brow, brow.data(), sizeof(int64_t) * (nb + 1),
                                 cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(H->d_bmat, bmat.data(), sizeof(int64_t) * (nb + 1),
                                 cudaMemcpyHostToDevice, s));
    k_dense_blocks<<<nb, 256, 0, s>>>(rp, ci, va, H->d_brow, H->d_bmat, dense, H->dev_status);
    AMG_LAUNCH_CHECK();
    if (largest_block(Lc, Lc.n) <= COARSE_SMALL) {  // one CUDA block per diagonal block
      k_cholesky<<<nb, 1024, 0, s>>>(H->d_brow, H->d_bmat, dense, H->Linv, H->LinvT,
                                     H->dev_status);
      AMG_LAUNCH_CHECK();
    } else {  // large blocks: blocked factorization over the whole GPU, block by block
      for (int b = 0; b < nb; ++b)
        AMG_TRY(chol_blocked(dense + bmat[b], brow[b + 1] - brow[b], H->Linv + bmat[b],
                             H->LinvT + bmat[b], H->dev_status, sms, s));
    }
    int st = read_status(H, s);  // synchronises: brow/bmat copies are done
    ar.release(dense);
    if (st < 0) return st;
  }
  // V-cycle work vectors (zeroed: the autotuner times kernels on them)
  const size_t vb = f32 ? sizeof(float) : sizeof(double);
  for (size_t l = 0; l < H->L.size(); ++l) {
    Level& L = H->L[l];
    L.vstore = VAL_F64;
    if (f32)
      L.vstore = (o.bf16_from_level > 0 && (int)l >= o.bf16_from_level) ? VAL_BF16 : VAL_F32;
    // nu_l = nu_0, or nu_0 * 2^l for the variable V-cycle (capped at 2^30)
    L.nu = o.variable_cycle ? (int64_t)o.smooth_sweeps << std::min<size_t>(l, 27)
                            : o.smooth_sweeps;
    for (void** v : {&L.b, &L.x, &L.r}) {
      AMG_TRY(ar.alloc(v, vb * (size_t)L.n));
      AMG_CUDA_TRY(cudaMemsetAsync(*v, 0, vb * (size_t)L.n, s));
    }
    if (L.nu > 1 && l + 1 < H->L.size())
      for (void** v : {&L.r2, &L.xp}) {
        AMG_TRY(ar.alloc(v, vb * (size_t)L.n));
        AMG_CUDA_TRY(cudaMemsetAsync(*v, 0, vb * (size_t)L.n, s));
      }
  }
  // sliced-ELL operators of every level, in the layout the options or the
  // autotuner choose
  const int64_t n0 = H->L[0].n;
  double *tb = nullptr, *tz = nullptr;  // FP64 level-0 vectors for timing
  if (o.autotune) {
    AMG_TRY(ar.alloc_n(&tb, n0));
    AMG_TRY(ar.alloc_n(&tz, n0));
    AMG_CUDA_TRY(cudaMemsetAsync(tb, 0, sizeof(double) * n0, s));
  }
  for (size_t l = 0; l < H->L.size(); ++l) {
    Level& L = H->L[l];
    const int64_t* rp = l == 0 ? A->rowptr : L.rowptr;
    const int32_t* ci = l == 0 ? A->col : L.col;
    const double* va = l == 0 ? A->val : L.val;
    const bool smooth = l + 1 < H->L.size();  // a level with a coarser one
    auto build = [&](Layout lay) -> int {
      const bool cmp = o.compress_columns != 0;
      AMG_TRY(sell_from_csr(ar, L.n, L.n, rp, ci, va, lay.C, lay.tpr, L.A, s,
                            H->batched ? &L.sys_off : nullptr, cmp));
      if (smooth) {
        AMG_TRY(build_ah(ar, L, sms, s));
        if (o.smooth_prolongator)
          AMG_TRY(build_smoothed_ops(ar, L, cmp, s));
        else
          AMG_TRY(build_ap(ar, L, rp, ci, va, cmp, sms, s));
      }
      return AMG_OK;
    };
    // threads per row: the option, else 32 / slice height, else by row length;
    // slice height: the option, else 32 / threads per row (always that for
    // batched systems, whose slices restart at every system)
    Layout lay;
    lay.tpr = o.threads_per_row > 0 ? o.threads_per_row
              : o.slice_height > 0  ? std::max(1, 32 / o.slice_height)
                                    : auto_tpr(L.n, L.nnz, L.vstore == VAL_F64);
    lay.C = o.slice_height > 0 && !H->batched ? o.slice_height : 32 / lay.tpr;
    if (like) {  // the assembled hierarchy's layout, tuned or not
      lay = {like->L[l].A.C, like->L[l].A.tpr};
    } else if (o.autotune && smooth && (l == 0 || L.n > o.tail_rows)) {
      // (levels that the persistent small-level launch runs are not tuned:
      // their per-level kernels never run in a V-cycle)
      const TuneKey key{L.n, (int)(10 * L.nnz / L.n), L.vstore, H->batched,
                        o.compress_columns != 0};
      if (!tune_lookup(key, &lay)) {
        const Layout def = lay;
        float best = 1e30f, def_ms = 1e30f;
        for (const Layout cand : tune_candidates(L.nnz >= 64 * L.n, H->batched)) {
          AMG_TRY(build(cand));
          // enough repetitions for about 2 ms of kernel time (small levels
          // take microseconds a launch), at least 3, at most 200
          float ms = 0.f;
          AMG_TRY(time_level(H, (int)l, 3, tb, tz, &ms, s));
          const int reps = (int)std::min(200.0f, std::max(3.0f, 2.0f / std::max(ms, 1e-4f)));
          if (reps > 3) AMG_TRY(time_level(H, (int)l, reps, tb, tz, &ms, s));
          if (cand.C == def.C && cand.tpr == def.tpr) def_ms = ms;
          if (ms < best) {
            best = ms;
            lay = cand;
          }
          release_level_ops(ar, L);
        }
        // the default layout unless another is clearly faster (3%)
        if (def_ms < 1e30f && best > 0.97f * def_ms) lay = def;
        tune_store(key, lay);
      }
    }
    AMG_TRY(build(lay));
  }
  ar.release(tb);
  ar.release(tz);
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  return AMG_OK;
}

}  // namespace amg
