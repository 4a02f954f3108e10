// Decoupled Vanek-Mandel-Brezina aggregation (Sec. 2.3, the VBM
// preconditioner of Sec. 3) on one GPU, where "decoupled" (no aggregate
// crosses a process boundary) changes nothing.
//
// Strong neighbourhood N_i = {i} + {j != i : |a_ij| >= theta sqrt(a_ii a_jj)},
// every edge's value read from row min(i, j), so the relation is symmetric.
// The sequential algorithm visits the rows in order and starts the aggregate
// N_i at every row whose whole neighbourhood is still free (phase 1), then
// adds every remaining row to the phase-1 aggregate of its most strongly
// coupled neighbour (phase 2; the smaller column on ties).  A row i is a
// phase-1 root exactly when no root r < i has N_r meeting N_i, so the roots
// are the first maximal set, in row order, of rows with pairwise disjoint
// neighbourhoods.  That set is found in rounds: an undecided row becomes a
// root once every row r < i within two strong steps is decided and none is a
// root, and is out as soon as one is.  Decisions are final and depend only on
// smaller rows, so the rounds reproduce the sequential result whatever order
// the threads run in.  With a symmetric pattern every row outside the
// phase-1 aggregates has a strong neighbour inside one, so nothing is left
// for the third phase of the sequential algorithm; a non-empty remainder is
// reported (AMG_ERR_UNSUPPORTED).  Aggregates are numbered by their roots.
#include "common.cuh"

namespace amg {

namespace {

constexpr int32_t VBM_UNDECIDED = 0;
constexpr int32_t VBM_ROOT = 1;
constexpr int32_t VBM_OUT = 2;

// strong[e]: entry e of row i is a strong neighbour j != i; mag[e] = |edge
// value| (0 where not strong).  Rounding as the oracle: one product, one
// square root, one product.
__global__ void k_vbm_strength(int64_t n, const int64_t* __restrict__ rowptr,
                               const int32_t* __restrict__ col, const double* __restrict__ val,
                               const double* __restrict__ diag, double theta,
                               uint8_t* __restrict__ strong, double* __restrict__ mag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double di = diag[i];
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int32_t j = col[e];
      double a = 0.0;
      bool st = false;
      if (j != i && edge_value(rowptr, col, val, (int32_t)i, j, val[e], &a)) {
        const double m = fabs(a);
        st = m >= __dmul_rn(theta, __dsqrt_rn(__dmul_rn(di, diag[j])));
        mag[e] = st ? m : 0.0;
      } else {
        mag[e] = 0.0;
      }
      strong[e] = st ? 1 : 0;
    }
  }
}

// Decision of row i from the current states: ROOT, OUT, or UNDECIDED (wait).
__device__ __forceinline__ int32_t vbm_decide(int32_t i, const int64_t* __restrict__ rowptr,
                                              const int32_t* __restrict__ col,
                                              const uint8_t* __restrict__ strong,
                                              const int32_t* state) {
  int32_t verdict = VBM_ROOT;
  // j runs over N_i (i itself first), r over N_j
  for (int64_t e = rowptr[i] - 1; e < rowptr[i + 1]; ++e) {
    int32_t j;
    if (e < rowptr[i]) {
      j = i;
    } else {
      if (!strong[e]) continue;
      j = col[e];
    }
    for (int64_t f = rowptr[j] - 1; f < rowptr[j + 1]; ++f) {
      int32_t r;
      if (f < rowptr[j]) {
        r = j;
      } else {
        if (!strong[f]) continue;
        r = col[f];
      }
      if (r >= i) continue;
      const int32_t st = __ldcg(state + r);  // other threads decide rows this round
      if (st == VBM_ROOT) return VBM_OUT;
      if (st == VBM_UNDECIDED) verdict = VBM_UNDECIDED;
    }
  }
  return verdict;
}

__global__ void k_vbm_round(const int32_t* __restrict__ wl, const int* __restrict__ nwl,
                            const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const uint8_t* __restrict__ strong, int32_t* state,
                            int32_t* __restrict__ wl_next, int* __restrict__ nwl_next,
                            int* rounds) {
  const int nw = *nwl;
  if (blockIdx.x == 0 && threadIdx.x == 0 && nw > 0) ++*rounds;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nw; t += gridDim.x * blockDim.x) {
    const int32_t i = wl[t];
    const int32_t v = vbm_decide(i, rowptr, col, strong, state);
    if (v == VBM_UNDECIDED)
      wl_next[atomicAdd(nwl_next, 1)] = i;
    else
      __stcg(state + i, v);
  }
}

__global__ void k_vbm_root_flags(int64_t n, const int32_t* __restrict__ state,
                                 int32_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = state[i] == VBM_ROOT ? 1 : 0;
}

// Phase 1: every root r labels N_r with its number (the neighbourhoods of
// roots are disjoint, so no row is written twice).
__global__ void k_vbm_cover(int64_t n, const int64_t* __restrict__ rowptr,
                            const int32_t* __restrict__ col, const uint8_t* __restrict__ strong,
                            const int32_t* __restrict__ state, const int32_t* __restrict__ id,
                            int32_t* __restrict__ agg) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (state[r] != VBM_ROOT) continue;
    const int32_t a = id[r];
    agg[r] = a;
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e)
      if (strong[e]) agg[col[e]] = a;
  }
}

// Phase 2 against the phase-1 labels agg1; rows without a strongly coupled
// labelled neighbour stay -1 and are counted in left.
__global__ void k_vbm_attach(int64_t n, const int64_t* __restrict__ rowptr,
                             const int32_t* __restrict__ col, const uint8_t* __restrict__ strong,
                             const double* __restrict__ mag, const int32_t* __restrict__ agg1,
                             int32_t* __restrict__ agg, int* left) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (agg1[i] >= 0) continue;
    int32_t best = -1;
    double bm = 0.0;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int32_t j = col[e];
      if (!strong[e] || agg1[j] < 0) continue;
      if (best < 0 || mag[e] > bm || (mag[e] == bm && j < best)) {
        best = j;
        bm = mag[e];
      }
    }
    if (best >= 0)
      agg[i] = agg1[best];
    else
      atomicAdd(left, 1);
  }
}

__global__ void k_vbm_sizes(int64_t n, const int32_t* __restrict__ agg, int32_t* cnt,
                            int* largest) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = atomicAdd(&cnt[agg[i]], 1) + 1;
    atomicMax(largest, c);
  }
}

}  // namespace

int vbm_aggregate(Arena& ar, int64_t n, const int64_t* rowptr, const int32_t* col,
                  const double* val, const double* diag, double theta, int32_t* agg, int64_t* nc,
                  int* stride, int num_sms, cudaStream_t s) {
  int64_t nnz = 0;  // entries are indexed as the row pointers give them, up to rowptr[n]
  AMG_CUDA_TRY(cudaMemcpyAsync(&nnz, rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  uint8_t* strong = nullptr;
  double* mag = nullptr;
  int32_t *state = nullptr, *wl = nullptr, *flag = nullptr, *id = nullptr, *agg1 = nullptr;
  int* cnt = nullptr;  // [0], [1]: worklist sizes; [2]: rounds; [3]: rows left; [4]: largest
  AMG_TRY(ar.alloc_n(&strong, nnz > 0 ? nnz : 1));
  AMG_TRY(ar.alloc_n(&mag, nnz > 0 ? nnz : 1));
  AMG_TRY(ar.alloc_n(&state, n));
  AMG_TRY(ar.alloc_n(&wl, 2 * n));
  AMG_TRY(ar.alloc_n(&cnt, 8));
  const int grid = grid_for(n, 256, num_sms, 8);
  k_vbm_strength<<<grid, 256, 0, s>>>(n, rowptr, col, val, diag, theta, strong, mag);
  AMG_LAUNCH_CHECK();
  AMG_CUDA_TRY(cudaMemsetAsync(state, 0, sizeof(int32_t) * n, s));
  const int hcnt[8] = {(int)n, 0, 0, 0, 0, 0, 0, 0};
  AMG_CUDA_TRY(cudaMemcpyAsync(cnt, hcnt, sizeof(hcnt), cudaMemcpyHostToDevice, s));
  k_iota<<<grid, 256, 0, s>>>(n, wl);
  AMG_LAUNCH_CHECK();
  int cur = 0;
  int rc = AMG_OK;
  int64_t launched = 0;
  for (;;) {
    // a batch of rounds between host checks; empty rounds exit immediately
    for (int r = 0; r < 8; ++r) {
      int32_t* w = wl + (int64_t)cur * n;
      int32_t* wn = wl + (int64_t)(1 - cur) * n;
      AMG_CUDA_TRY(cudaMemsetAsync(cnt + 1 - cur, 0, sizeof(int), s));
      k_vbm_round<<<grid, 256, 0, s>>>(w, cnt + cur, rowptr, col, strong, state, wn,
                                       cnt + 1 - cur, cnt + 2);
      AMG_LAUNCH_CHECK();
      cur = 1 - cur;
    }
    launched += 8;
    int h[8];
    AMG_CUDA_TRY(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (h[cur] == 0) break;
    if (launched > n + 64) {  // each round decides at least the smallest undecided row
      rc = AMG_ERR_DEVICE_CHECK;
      break;
    }
  }
  if (rc == AMG_OK) {
    AMG_TRY(ar.alloc_n(&flag, n));
    AMG_TRY(ar.alloc_n(&id, n));
    AMG_TRY(ar.alloc_n(&agg1, n));
    k_vbm_root_flags<<<grid, 256, 0, s>>>(n, state, flag);
    AMG_LAUNCH_CHECK();
    int64_t roots = 0;
    AMG_TRY(scan_exclusive_i32(ar, flag, id, n, &roots, s));
    AMG_CUDA_TRY(cudaMemsetAsync(agg1, 0xFF, sizeof(int32_t) * n, s));
    k_vbm_cover<<<grid, 256, 0, s>>>(n, rowptr, col, strong, state, id, agg1);
    AMG_LAUNCH_CHECK();
    AMG_CUDA_TRY(cudaMemcpyAsync(agg, agg1, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    k_vbm_attach<<<grid, 256, 0, s>>>(n, rowptr, col, strong, mag, agg1, agg, cnt + 3);
    AMG_LAUNCH_CHECK();
    int left = 0;
    AMG_CUDA_TRY(cudaMemcpyAsync(&left, cnt + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (left > 0) {
      rc = AMG_ERR_UNSUPPORTED;
    } else {
      int32_t* sizes = nullptr;
      AMG_TRY(ar.alloc_n(&sizes, roots > 0 ? roots : 1));
      AMG_CUDA_TRY(cudaMemsetAsync(sizes, 0, sizeof(int32_t) * (roots > 0 ? roots : 1), s));
      k_vbm_sizes<<<grid, 256, 0, s>>>(n, agg, sizes, cnt + 4);
      AMG_LAUNCH_CHECK();
      int largest = 0;
      AMG_CUDA_TRY(cudaMemcpyAsync(&largest, cnt + 4, sizeof(int), cudaMemcpyDeviceToHost, s));
      AMG_CUDA_TRY(cudaStreamSynchronize(s));
      ar.release(sizes);
      int st = 1;
      while (st < largest) st <<= 1;
      *stride = st;
      *nc = roots;
    }
  }
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  for (void* p : {(void*)strong, (void*)mag, (void*)state, (void*)wl, (void*)cnt, (void*)flag,
                  (void*)id, (void*)agg1})
    ar.release(p);
  return rc;
}

}  // namespace amg
