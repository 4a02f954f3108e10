// Allocation-free pairwise matching: amg_pairwise_match_noalloc.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured, applications whose device memory belongs to a pool or
// framework that forbids outside allocations, and real-time loops that must
// not allocate (or risk an allocator stall) after start-up.  For them this
// entry point runs the same matching kernels as amg_pairwise_match, with all
// of its scratch (diagonal, pointers, frontier flags and lists, counters) in
// one file-scope __device__ array of fixed size instead of cudaMalloc'ed
// buffers.  The caller still passes the matrix and the output array.
//
// The array is sized for AMG_NOALLOC_MAX_ROWS rows (24 bytes a row, 6 MiB);
// every GPU that loads this library holds it until the process exits.  Its
// device address is looked up once per device (cudaGetSymbolAddress) by the
// first call made with that device current.  All calls share the array, so
// calls that overlap on the GPU (different streams or host threads) race.
#include <mutex>

#include "common.cuh"

namespace amg {

constexpr int64_t NA_ROWS = AMG_NOALLOC_MAX_ROWS;
constexpr size_t NA_DIAG = 0;                                      // double[rows]
constexpr size_t NA_CAND = NA_DIAG + sizeof(double) * NA_ROWS;     // int32[rows]
constexpr size_t NA_FLAG = NA_CAND + sizeof(int32_t) * NA_ROWS;    // int32[rows]
constexpr size_t NA_WL = NA_FLAG + sizeof(int32_t) * NA_ROWS;      // int32[2 * rows]
constexpr size_t NA_CNT = NA_WL + sizeof(int32_t) * 2 * NA_ROWS;   // int[4]
constexpr size_t NA_BYTES = NA_CNT + 256;

static __device__ __align__(256) unsigned char g_match_scratch[NA_BYTES];

static std::mutex g_scratch_mu;
static unsigned char* g_scratch_ptr[256];  // per device; host-side lookup result

// Device address of g_match_scratch on the current device (looked up once).
static int scratch_base(unsigned char** base) {
  int dev = 0;
  AMG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return AMG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    AMG_CUDA_TRY(cudaGetSymbolAddress(&p, g_match_scratch));
    g_scratch_ptr[dev] = (unsigned char*)p;
  }
  *base = g_scratch_ptr[dev];
  return AMG_OK;
}

__global__ void k_noalloc_counts(int* cnt, int n) {
  if (threadIdx.x == 0) {
    cnt[0] = n;  // the first frontier holds every row
    cnt[1] = 0;
    cnt[2] = 0;  // rounds with a non-empty frontier
    cnt[3] = 0;
  }
}

static int match_noalloc(const amg_csr* A, int32_t* mate, int* rounds_out, cudaStream_t s) {
  unsigned char* base = nullptr;
  AMG_TRY(scratch_base(&base));
  const int64_t n = A->n;
  double* diag = (double*)(base + NA_DIAG);
  int32_t* cand = (int32_t*)(base + NA_CAND);
  int32_t* flag = (int32_t*)(base + NA_FLAG);
  int32_t* wl = (int32_t*)(base + NA_WL);
  int* cnt = (int*)(base + NA_CNT);
  int dev = 0, sms = 0;
  AMG_CUDA_TRY(cudaGetDevice(&dev));
  AMG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = grid_for(n, 256, sms, 8);
  k_l1_diag<<<grid, 256, 0, s>>>(n, A->rowptr, A->col, A->val, nullptr, diag);
  AMG_LAUNCH_CHECK();
  // the array keeps the previous call's contents: reset what must start at zero
  AMG_CUDA_TRY(cudaMemsetAsync(mate, 0xFF, sizeof(int32_t) * n, s));
  AMG_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int32_t) * n, s));
  k_noalloc_counts<<<1, 32, 0, s>>>(cnt, (int)n);
  AMG_LAUNCH_CHECK();
  k_iota<<<grid, 256, 0, s>>>(n, wl);
  AMG_LAUNCH_CHECK();
  int cur = 0;
  int rc = AMG_OK;
  int64_t launched = 0;
  for (;;) {
    for (int r = 0; r < 8; ++r) {
      int32_t* w = wl + (int64_t)cur * NA_ROWS;
      int32_t* wn = wl + (int64_t)(1 - cur) * NA_ROWS;
      k_match_cand<<<grid, 256, 0, s>>>(w, cnt + cur, A->rowptr, A->col, A->val, diag, mate,
                                        cand, flag, cnt + 2);
      AMG_LAUNCH_CHECK();
      k_match_commit<<<grid, 256, 0, s>>>(w, cnt + cur, cand, mate);
      AMG_LAUNCH_CHECK();
      AMG_CUDA_TRY(cudaMemsetAsync(cnt + 1 - cur, 0, sizeof(int), s));
      k_match_expand<<<grid, 256, 0, s>>>(w, cnt + cur, A->rowptr, A->col, mate, flag, wn,
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

}  // namespace amg

extern "C" int amg_pairwise_match_noalloc(const amg_csr* A, int32_t* mate, int* rounds,
                                          amg_stream_t stream) {
  if (!A || A->n <= 0 || A->nnz < A->n || !A->rowptr || !A->col || !A->val || !mate)
    return AMG_ERR_ARG;
  if (A->n > AMG_NOALLOC_MAX_ROWS) return AMG_ERR_UNSUPPORTED;
  return amg::match_noalloc(A, mate, rounds, (cudaStream_t)stream);
}
