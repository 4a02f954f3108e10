// Allocation, error notes, grid sizing and exclusive scans.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"

namespace amg {

static std::atomic<long> g_fail_after{-1};  // test hook: fail the k-th allocation

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  if (getenv("AMG_VERBOSE"))
    fprintf(stderr, "[amg] CUDA error %d (%s) at %s:%d: %s\n", (int)e, cudaGetErrorString(e), file,
            line, what);
}

int Arena::alloc(void** p, size_t bytes) {
  *p = nullptr;
  long k = g_fail_after.load();
  if (k >= 0) {
    if (k == 0) {
      g_fail_after.store(-1);
      return AMG_ERR_OOM;
    }
    g_fail_after.store(k - 1);
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? AMG_ERR_OOM : AMG_ERR_CUDA;
  }
  blocks.push_back(*p);
  return AMG_OK;
}

void Arena::release(void* p) {
  if (!p) return;
  auto it = std::find(blocks.begin(), blocks.end(), p);
  if (it != blocks.end()) {
    cudaFree(p);
    blocks.erase(it);
  }
}

void Arena::release_all() {
  for (void* p : blocks) cudaFree(p);
  blocks.clear();
}

int grid_for(int64_t work_items, int threads, int num_sms, int blocks_per_sm) {
  int64_t need = (work_items + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms * blocks_per_sm;
  if (need < 1) need = 1;
  return (int)std::min(need, cap);
}

// ------------------------------------------------------------------ scans
// Three phases over tiles of SCAN_TILE elements: tile sums, a single-block
// scan of the tile sums (looping over chunks), then each tile rescans itself.

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T v, T* total) {
  __shared__ T warp_tot[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    T t = warp_tot[lane];
    T s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T u = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += u;
    }
    warp_tot[lane] = s - t;  // exclusive warp offsets
    if (lane == 31) *total = s;
  }
  __syncthreads();
  T r = warp_tot[w] + inc - v;
  __syncthreads();
  return r;
}

template <typename Tin, typename Tout>
__global__ void k_tile_sums(const Tin* in, int64_t n, Tout* sums) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  Tout v = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
    if (i < n) v += (Tout)in[i];
  }
  __shared__ Tout tot;
  block_exclusive_scan<Tout>(v, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scan_sums(T* sums, int64_t m, T* grand) {
  __shared__ T tot;
  T carry = 0;
  for (int64_t base = 0; base < m; base += SCAN_THREADS) {
    int64_t i = base + threadIdx.x;
    T v = i < m ? sums[i] : 0;
    T ex = block_exclusive_scan<T>(v, &tot);
    if (i < m) sums[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *grand = carry;
}

template <typename Tin, typename Tout>
__global__ void k_tile_scan(const Tin* in, int64_t n, const Tout* offs, Tout* out) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  Tout loc[SCAN_ITEMS];
  Tout v = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
    loc[k] = i < n ? (Tout)in[i] : 0;
    v += loc[k];
  }
  __shared__ Tout tot;
  Tout ex = block_exclusive_scan<Tout>(v, &tot) + offs[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
    if (i < n) out[i] = ex;
    ex += loc[k];
  }
}

template <typename T>
static int scan_impl(Arena& ar, const T* in, T* out, int64_t n, int64_t* total, cudaStream_t s) {
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles < 1) tiles = 1;
  T* sums = nullptr;
  AMG_TRY(ar.alloc_n(&sums, tiles + 1));
  if (n > 0) {
    k_tile_sums<T, T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums);
    AMG_LAUNCH_CHECK();
  }
  k_scan_sums<T><<<1, SCAN_THREADS, 0, s>>>(sums, n > 0 ? tiles : 0, sums + tiles);
  AMG_LAUNCH_CHECK();
  if (n > 0) {
    k_tile_scan<T, T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums, out);
    AMG_LAUNCH_CHECK();
  }
  int rc = AMG_OK;
  if (total) {
    T t = 0;
    cudaError_t e = cudaMemcpyAsync(&t, sums + tiles, sizeof(T), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = AMG_ERR_CUDA;
    *total = (int64_t)t;
  }
  ar.release(sums);
  return rc;
}

int scan_exclusive_i32(Arena& ar, const int32_t* in, int32_t* out, int64_t n, int64_t* total,
                       cudaStream_t s) {
  return scan_impl<int32_t>(ar, in, out, n, total, s);
}

int scan_exclusive_i64(Arena& ar, const int64_t* in, int64_t* out, int64_t n, int64_t* total,
                       cudaStream_t s) {
  return scan_impl<int64_t>(ar, in, out, n, total, s);
}

}  // namespace amg

extern "C" int amg_debug_fail_alloc_after(long count) {
  amg::g_fail_after.store(count);
  return AMG_OK;
}
