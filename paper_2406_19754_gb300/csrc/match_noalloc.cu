// Allocation-free pairwise matching: amg_pairwise_match_noalloc.
//
// Some callers cannot call cudaMalloc: applications whose device memory
// belongs to a pool or framework that forbids outside allocations, and
// real-time loops that must not allocate (or risk an allocator stall) after
// start-up.  For them this entry point runs the same matching kernels as
// amg_pairwise_match, with all of its scratch (diagonal, pointers, frontier
// flags and lists, counters) in one file-scope __device__ array of fixed size
// instead of cudaMalloc'ed buffers.  The caller still passes the matrix and
// the output array.
//
// The array is sized for AMG_NOALLOC_MAX_ROWS rows (24 bytes a row, 6 MiB);
// every GPU that loads this library holds it until the process exits.  Its
// device address is looked up once per device (cudaGetSymbolAddress) by the
// first call made with that device current, and kept: after cudaDeviceReset
// the kept address belongs to a context that no longer exists, so the entry
// point must not be called on a device that was reset in this process.  All
// calls share the array, so calls that overlap on the GPU (different streams
// or host threads) race.
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
  k_l1_diag<<<grid_for(n, 256, sms, 8), 256, 0, s>>>(n, A->rowptr, A->col, A->val, nullptr,
                                                    diag);
  AMG_LAUNCH_CHECK();
  // the same round loop as amg_pairwise_match, on the static scratch (its
  // two frontiers NA_ROWS entries apart); it clears what must start at zero
  return match_round_loop(n, A->rowptr, A->col, A->val, diag, mate, cand, flag, wl, NA_ROWS,
                          cnt, rounds_out, sms, s);
}

}  // namespace amg

extern "C" int amg_pairwise_match_noalloc(const amg_csr* A, int32_t* mate, int* rounds,
                                          amg_stream_t stream) {
  const int rc = amg::check_csr(A);
  if (rc < 0) return rc;
  if (!mate) return AMG_ERR_ARG;
  if (A->n > AMG_NOALLOC_MAX_ROWS) return AMG_ERR_UNSUPPORTED;
  return amg::match_noalloc(A, mate, rounds, (cudaStream_t)stream);
}
