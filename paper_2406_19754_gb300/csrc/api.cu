// C-ABI entry points declared in include/amg.h: argument checks, handle
// lifecycle, and dispatch into the setup, V-cycle and PCG drivers.
#include <string.h>

#include <utility>

#include "common.cuh"

using namespace amg;

namespace amg {

int check_csr(const amg_csr* A) {
  if (!A || A->n <= 0 || A->nnz < A->n || !A->rowptr || !A->col || !A->val) return AMG_ERR_ARG;
  if (A->n > (int64_t)0x7fffffff) return AMG_ERR_UNSUPPORTED;
  return AMG_OK;
}

}  // namespace amg

extern "C" {

int amg_default_options(amg_options* o) {
  if (!o) return AMG_ERR_ARG;
  memset(o, 0, sizeof(*o));
  o->sweeps = 2;
  o->max_levels = 30;
  o->max_coarse = 200;
  o->stall_ratio = 0.9;
  o->max_dense = 8192;
  o->precision = AMG_PREC_F64;
  o->bf16_from_level = 0;
  o->slice_height = 0;
  o->threads_per_row = 0;
  o->autotune = 0;
  o->tail_rows = 1024;
  o->smooth_sweeps = 1;
  o->variable_cycle = 0;
  o->coarse_solver = 0;
  o->coarse_maxit = 40;
  o->coarse_tol = 1e-4;
  o->compress_columns = 0;
  o->smooth_prolongator = 0;
  o->aggregation = 0;
  o->vbm_theta = 0.01;
  o->prolongator_filter = 0.0;
  o->stream_ring = 1;
  return AMG_OK;
}

int pcg_default_options(pcg_options* o) {
  if (!o) return AMG_ERR_ARG;
  memset(o, 0, sizeof(*o));
  o->tol = 1e-8;
  o->maxit = 500;
  o->beta_form = PCG_BETA_AUTO;
  o->use_graph = 1;
  return AMG_OK;
}

const char* amg_status_string(int s) {
  switch (s) {
    case AMG_OK: return "ok";
    case AMG_NOT_CONVERGED: return "not converged (maxit reached)";
    case AMG_ERR_ARG: return "invalid argument";
    case AMG_ERR_NOT_SPD: return "matrix not symmetric positive definite (coarse Cholesky)";
    case AMG_ERR_BREAKDOWN: return "PCG breakdown: p^T A p <= 0";
    case AMG_ERR_NAN: return "NaN or Inf in a PCG scalar";
    case AMG_ERR_CUDA: return "CUDA error";
    case AMG_ERR_OOM: return "device allocation failed";
    case AMG_ERR_DEVICE_CHECK: return "device-side check failed";
    case AMG_ERR_UNSUPPORTED: return "input outside implemented limits";
    default: return "unknown status";
  }
}

static int check_options(const amg_options& o) {
  if (o.sweeps < 1 || o.sweeps > 3) return AMG_ERR_ARG;
  if (o.max_levels < 1 || o.max_coarse < 1 || o.max_dense < 1 || o.max_dense > 16384)
    return AMG_ERR_ARG;
  if (!(o.stall_ratio > 0.0 && o.stall_ratio <= 1.0)) return AMG_ERR_ARG;
  if (o.precision != AMG_PREC_F64 && o.precision != AMG_PREC_F32) return AMG_ERR_ARG;
  if (o.bf16_from_level < 0 || o.tail_rows < 0) return AMG_ERR_ARG;
  if (o.compress_columns != 0 && o.compress_columns != 1) return AMG_ERR_ARG;
  if (o.smooth_prolongator != 0 && o.smooth_prolongator != 1) return AMG_ERR_ARG;
  if (o.aggregation != 0 && o.aggregation != 1) return AMG_ERR_ARG;
  if (!(o.vbm_theta >= 0.0 && o.vbm_theta < 1.0)) return AMG_ERR_ARG;
  if (!(o.prolongator_filter >= 0.0 && o.prolongator_filter < 1.0)) return AMG_ERR_ARG;
  if (o.stream_ring < 0 || o.stream_ring > 4) return AMG_ERR_ARG;
  if (o.smooth_sweeps < 1 || o.smooth_sweeps > 8) return AMG_ERR_ARG;
  if (o.variable_cycle != 0 && o.variable_cycle != 1) return AMG_ERR_ARG;
  if (o.coarse_solver != 0 && o.coarse_solver != 1) return AMG_ERR_ARG;
  if (o.coarse_maxit < 0 || o.coarse_maxit > 100000 || !(o.coarse_tol >= 0.0))
    return AMG_ERR_ARG;
  const int C = o.slice_height, t = o.threads_per_row;
  if (C != 0 && C != 1 && C != 2 && C != 4 && C != 8 && C != 16 && C != 32 && C != 64)
    return AMG_ERR_ARG;
  if (t != 0 && t != 1 && t != 2 && t != 4 && t != 8 && t != 16 && t != 32) return AMG_ERR_ARG;
  return AMG_OK;
}

static void destroy(amg_handle* H) {
  if (!H) return;
  multi_free(H);
  tg_free(H);
  if (H->batch.sc_host) cudaFreeHost(H->batch.sc_host);
  if (H->bgraph) cudaGraphExecDestroy(H->bgraph);
  if (H->graph) cudaGraphExecDestroy(H->graph);
  if (H->loop) cudaGraphExecDestroy(H->loop);
  if (H->bloop) cudaGraphExecDestroy(H->bloop);
  if (H->cap_stream) cudaStreamDestroy(H->cap_stream);
  if (H->ev0) cudaEventDestroy(H->ev0);
  if (H->ev1) cudaEventDestroy(H->ev1);
  if (H->sc_host) cudaFreeHost(H->sc_host);
  H->arena.release_all();
  delete H;
}

// Order-independent fingerprint of a CSR sparsity pattern: the wrapping sum
// of splitmix64 hashes of (row, row pointer) and (position, column).
__global__ void k_pattern_hash(int64_t n, const int64_t* rowptr, const int32_t* col,
                               unsigned long long* out) {
  const int64_t nnz = rowptr[n] - rowptr[0];
  unsigned long long h = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n + nnz;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i <= n)
      h += mix64(((uint64_t)i << 40) ^ (uint64_t)(rowptr[i] - rowptr[0]));
    else
      h += mix64(0x9E3779B97F4A7C15ull ^ ((uint64_t)(i - n - 1) << 32) ^
                 (uint64_t)(uint32_t)col[rowptr[0] + (i - n - 1)]);
  }
  h = warp_sum(h);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, h);
}

static int pattern_hash(const amg_csr* A, unsigned long long* h, cudaStream_t s, int num_sms) {
  unsigned long long* d = nullptr;
  AMG_CUDA_TRY(cudaMallocAsync((void**)&d, sizeof(*d), s));
  AMG_CUDA_TRY(cudaMemsetAsync(d, 0, sizeof(*d), s));
  k_pattern_hash<<<grid_for(A->n + A->nnz + 1, 256, num_sms, 4), 256, 0, s>>>(A->n, A->rowptr,
                                                                               A->col, d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(*h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(d, s);
  AMG_CUDA_TRY(e);
  return AMG_OK;
}

static int create(const amg_csr* A, const amg_options* opt, cudaStream_t s, amg_handle** out,
                  int nsys = 0, const amg_csr* systems = nullptr,
                  const amg_handle* like = nullptr) {
  amg_handle* H = new amg_handle();
  *out = H;
  if (opt)
    H->opt = *opt;
  else
    amg_default_options(&H->opt);
  AMG_TRY(check_options(H->opt));
  amg_csr cat;
  int64_t* cat_rp = nullptr;
  int32_t* cat_ci = nullptr;
  double* cat_va = nullptr;
  if (systems && H->opt.coarse_solver != 0) return AMG_ERR_UNSUPPORTED;
  if (H->opt.smooth_prolongator && (systems || H->opt.autotune)) return AMG_ERR_UNSUPPORTED;
  if (systems) {  // batched: one block-diagonal matrix with system-aligned slices
    int dev = 0, sms = 0;
    AMG_CUDA_TRY(cudaGetDevice(&dev));
    AMG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    AMG_TRY(concat_systems(H->arena, nsys, systems, &cat, &cat_rp, &cat_ci, &cat_va,
                           H->sys_off0, sms, s));
    H->batched = true;
    H->nsys = nsys;
    A = &cat;
  }
  AMG_CUDA_TRY(cudaGetDevice(&H->device));
  AMG_CUDA_TRY(cudaDeviceGetAttribute(&H->num_sms, cudaDevAttrMultiProcessorCount, H->device));
  AMG_CUDA_TRY(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
  AMG_CUDA_TRY(cudaEventCreate(&H->ev0));
  AMG_CUDA_TRY(cudaEventCreate(&H->ev1));
  AMG_CUDA_TRY(cudaMallocHost((void**)&H->sc_host, sizeof(PcgScalars)));
  Arena& ar = H->arena;
  AMG_TRY(ar.alloc_n(&H->dev_status, 1));
  AMG_CUDA_TRY(cudaMemsetAsync(H->dev_status, 0, sizeof(int), s));
  AMG_TRY(ar.alloc_n(&H->wait_fail, 1));
  AMG_CUDA_TRY(cudaMemsetAsync(H->wait_fail, 0, sizeof(int), s));
  H->red.max_blocks = H->num_sms * 16;
  AMG_TRY(ar.alloc_n(&H->red.partials, (int64_t)H->red.max_blocks * 4));
  AMG_TRY(ar.alloc_n(&H->red.ticket, 1));
  AMG_CUDA_TRY(cudaMemsetAsync(H->red.ticket, 0, sizeof(unsigned), s));
  AMG_TRY(ar.alloc_n(&H->sc, 1));
  AMG_CUDA_TRY(cudaMemsetAsync(H->sc, 0, sizeof(PcgScalars), s));
  if (!systems) AMG_TRY(pattern_hash(A, &H->pattern, s, H->num_sms));
  AMG_TRY(setup_hierarchy(H, A, s, like));
  const int64_t n = A->n;
  AMG_TRY(ar.alloc_n(&H->r, n));
  AMG_TRY(ar.alloc_n(&H->z, n));
  AMG_TRY(ar.alloc_n(&H->p, n));
  AMG_TRY(ar.alloc_n(&H->q, n));
  if (H->opt.precision == AMG_PREC_F32 && H->L.size() > 1)
    AMG_TRY(ar.alloc_n(&H->r32, n));
  if (H->batched) {
    AMG_TRY(batch_init(H, s));
    ar.release(cat_rp);  // the hierarchy keeps its own copies
    ar.release(cat_ci);
    ar.release(cat_va);
  }
  AMG_TRY(tail_init(H, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  return AMG_OK;
}

int amg_setup(const amg_csr* A, const amg_options* opt, amg_stream_t stream, amg_handle** H) {
  if (!H) return AMG_ERR_ARG;
  *H = nullptr;
  int rc = check_csr(A);
  if (rc < 0) return rc;
  amg_handle* h = nullptr;
  rc = create(A, opt, (cudaStream_t)stream, &h);
  if (rc < 0) {
    cudaStreamSynchronize((cudaStream_t)stream);
    destroy(h);
    return rc;
  }
  *H = h;
  return AMG_OK;
}

int amg_destroy(amg_handle* H) {
  destroy(H);
  return AMG_OK;
}

int amg_update_values(amg_handle* H, const amg_csr* A, amg_stream_t stream) {
  if (!H) return AMG_ERR_ARG;
  if (H->batched) return AMG_ERR_UNSUPPORTED;
  int rc = check_csr(A);
  if (rc < 0) return rc;
  if (A->n != H->L[0].n || A->nnz != H->L[0].nnz) return AMG_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long h = 0;
  rc = pattern_hash(A, &h, s, H->num_sms);
  if (rc < 0) return rc;
  if (h != H->pattern) return AMG_ERR_ARG;
  amg_handle* T = nullptr;
  rc = create(A, &H->opt, s, &T, 0, nullptr, H);
  if (rc < 0) {
    cudaStreamSynchronize(s);
    destroy(T);
    return rc;
  }
  std::swap(*H, *T);  // H keeps its address; T now holds the old hierarchy
  destroy(T);
  return AMG_OK;
}

int amg_setup_batch(int nsys, const amg_csr* A, const amg_options* opt, amg_stream_t stream,
                    amg_handle** H) {
  if (!H) return AMG_ERR_ARG;
  *H = nullptr;
  if (nsys <= 0 || !A) return AMG_ERR_ARG;
  for (int k = 0; k < nsys; ++k) {
    int rc = check_csr(&A[k]);
    if (rc < 0) return rc;
  }
  amg_handle* h = nullptr;
  int rc = create(nullptr, opt, (cudaStream_t)stream, &h, nsys, A);
  if (rc < 0) {
    cudaStreamSynchronize((cudaStream_t)stream);
    destroy(h);
    return rc;
  }
  *H = h;
  return AMG_OK;
}

int amg_batch_info(const amg_handle* H, int* nsys, int64_t* row_offsets) {
  if (!H || !nsys) return AMG_ERR_ARG;
  *nsys = H->batched ? H->nsys : 1;
  if (row_offsets) {
    if (H->batched)
      for (int k = 0; k <= H->nsys; ++k) row_offsets[k] = H->sys_off0[k];
    else {
      row_offsets[0] = 0;
      row_offsets[1] = H->L[0].n;
    }
  }
  return AMG_OK;
}

int pcg_solve_batch(amg_handle* H, const double* b, double* x, const pcg_options* o,
                    pcg_stats* st, amg_stream_t stream) {
  if (!H || !b || !x || !H->batched) return AMG_ERR_ARG;
  pcg_options def;
  pcg_default_options(&def);
  const pcg_options* op = o ? o : &def;
  if (op->maxit < 0 || !(op->tol >= 0.0)) return AMG_ERR_ARG;
  if (op->beta_form < PCG_BETA_AUTO || op->beta_form > PCG_BETA_FLEXIBLE) return AMG_ERR_ARG;
  if (op->res_history || op->x_history) return AMG_ERR_ARG;  // per-system histories: not kept
  if (op->use_graph < 0 || op->use_graph > 2) return AMG_ERR_ARG;
  return pcg_batch_run(H, b, x, op, st, (cudaStream_t)stream);
}

int amg_set_smoother_weights(amg_handle* H, const float* omega, amg_stream_t stream) {
  if (!H) return AMG_ERR_ARG;
  return set_level0_weights(H, omega, (cudaStream_t)stream);
}

int amg_vcycle_apply(const amg_handle* H, const double* r, double* z, amg_stream_t stream) {
  if (!H || !r || !z || (const double*)z == r) return AMG_ERR_ARG;
  return vcycle_run(H, r, z, 0, nullptr, (cudaStream_t)stream);
}

int amg_vcycle_profile(const amg_handle* H, const double* r, double* z, amg_kernel_time* out,
                       int max_out, int* count, amg_stream_t stream) {
  if (!H || !r || !z || (const double*)z == r || max_out < 0 || (max_out > 0 && !out))
    return AMG_ERR_ARG;
  return vcycle_profile(H, r, z, out, max_out, count, (cudaStream_t)stream);
}

int amg_debug_convert(const double* in64, float* out32, const float* in32, double* out64,
                      int64_t n, amg_stream_t stream) {
  if (n < 0 || (!in64) != (!out32) || (!in32) != (!out64)) return AMG_ERR_ARG;
  return debug_convert(in64, out32, in32, out64, n, (cudaStream_t)stream);
}

int amg_spmv(const amg_handle* H, int level, double alpha, const double* x, double beta,
             double* y, amg_stream_t stream) {
  if (!H || level < 0 || level >= (int)H->L.size() || !x || !y || (const double*)y == x)
    return AMG_ERR_ARG;
  return sell_spmv64(H->L[level].A, alpha, x, beta, y, H->num_sms, (cudaStream_t)stream);
}

int pcg_solve(amg_handle* H, const double* b, double* x, const pcg_options* o, pcg_stats* st,
              amg_stream_t stream) {
  if (!H || !b || !x) return AMG_ERR_ARG;
  pcg_options def;
  pcg_default_options(&def);
  const pcg_options* op = o ? o : &def;
  if (op->maxit < 0 || !(op->tol >= 0.0)) return AMG_ERR_ARG;
  if (op->beta_form < PCG_BETA_AUTO || op->beta_form > PCG_BETA_FLEXIBLE) return AMG_ERR_ARG;
  if (op->use_graph < 0 || op->use_graph > 2) return AMG_ERR_ARG;
  return pcg_run(H, b, x, op, st, (cudaStream_t)stream);
}

int amg_vcycle_apply_multi(amg_handle* H, int nrhs, const double* R, double* Z,
                           amg_stream_t stream) {
  if (!H || !R || !Z || (const double*)Z == R || nrhs < 1 || nrhs > 64) return AMG_ERR_ARG;
  if (H->L.size() < 2 || H->L[0].A.row0 || H->opt.smooth_prolongator) return AMG_ERR_UNSUPPORTED;
  return vcycle_multi(H, nrhs, R, Z, (cudaStream_t)stream);
}

int pcg_solve_multi(amg_handle* H, int nrhs, const double* B, double* X, const pcg_options* o,
                    pcg_stats* st, amg_stream_t stream) {
  if (!H || !B || !X || nrhs < 1 || nrhs > 64) return AMG_ERR_ARG;
  if (H->L.size() < 2 || H->L[0].A.row0 || H->opt.smooth_prolongator) return AMG_ERR_UNSUPPORTED;
  pcg_options def;
  pcg_default_options(&def);
  const pcg_options* op = o ? o : &def;
  if (op->maxit < 0 || !(op->tol >= 0.0)) return AMG_ERR_ARG;
  if (op->beta_form < PCG_BETA_AUTO || op->beta_form > PCG_BETA_FLEXIBLE) return AMG_ERR_ARG;
  if (op->res_history || op->x_history) return AMG_ERR_ARG;
  return pcg_multi_run(H, nrhs, B, X, op, st, (cudaStream_t)stream);
}

int amg_twogrid_loss(amg_handle* H, int nsamples, int ncycles, const double* e0, double* loss,
                     float* domega, amg_stream_t stream) {
  if (!H || nsamples < 1 || ncycles < 1 || !e0 || !loss) return AMG_ERR_ARG;
  if (H->opt.smooth_prolongator) return AMG_ERR_UNSUPPORTED;
  return twogrid_loss(H, nsamples, ncycles, e0, loss, domega, (cudaStream_t)stream);
}

int amg_num_levels(const amg_handle* H, int* levels) {
  if (!H || !levels) return AMG_ERR_ARG;
  *levels = (int)H->L.size();
  return AMG_OK;
}

int amg_level_info(const amg_handle* H, int level, int64_t* n, int64_t* nnz) {
  if (!H || level < 0 || level >= (int)H->L.size()) return AMG_ERR_ARG;
  if (n) *n = H->L[level].n;
  if (nnz) *nnz = H->L[level].nnz;
  return AMG_OK;
}

int amg_level_layout(const amg_handle* H, int level, int ap, amg_layout* out) {
  if (!H || !out || level < 0 || level >= (int)H->L.size() || ap < 0 || ap > 3)
    return AMG_ERR_ARG;
  if (ap && level == (int)H->L.size() - 1) return AMG_ERR_ARG;
  if (ap >= 2 && !H->opt.smooth_prolongator) return AMG_ERR_ARG;
  const Level& L = H->L[level];
  const Sell& M = ap == 0 ? L.A : ap == 1 ? L.AP : ap == 2 ? L.P : L.R;
  out->slice_height = M.C;
  out->threads_per_row = M.tpr;
  out->slots = M.nnz_pad;
  out->compressed = M.d16 ? 1 : 0;
  return AMG_OK;
}

int amg_level_export(const amg_handle* H, int level, int64_t* rowptr, int32_t* col, double* val,
                     int32_t* agg, double* sscale, amg_stream_t stream) {
  if (!H || level < 0 || level >= (int)H->L.size()) return AMG_ERR_ARG;
  const Level& L = H->L[level];
  cudaStream_t s = (cudaStream_t)stream;
  if ((rowptr || col || val) && level == 0) return AMG_ERR_ARG;
  if (agg && !L.agg) return AMG_ERR_ARG;
  if (rowptr)
    AMG_CUDA_TRY(cudaMemcpyAsync(rowptr, L.rowptr, sizeof(int64_t) * (L.n + 1),
                                 cudaMemcpyDeviceToDevice, s));
  if (col)
    AMG_CUDA_TRY(cudaMemcpyAsync(col, L.col, sizeof(int32_t) * L.nnz, cudaMemcpyDeviceToDevice, s));
  if (val)
    AMG_CUDA_TRY(cudaMemcpyAsync(val, L.val, sizeof(double) * L.nnz, cudaMemcpyDeviceToDevice, s));
  if (agg)
    AMG_CUDA_TRY(cudaMemcpyAsync(agg, L.agg, sizeof(int32_t) * L.n, cudaMemcpyDeviceToDevice, s));
  if (sscale)
    AMG_CUDA_TRY(cudaMemcpyAsync(sscale, L.s64, sizeof(double) * L.n, cudaMemcpyDeviceToDevice, s));
  return AMG_OK;
}

int amg_level_prolongator(const amg_handle* H, int level, int64_t* rowptr, int32_t* col,
                          double* val, int64_t* nnz, double* w, amg_stream_t stream) {
  if (!H || level < 0 || level + 1 >= (int)H->L.size() || !H->opt.smooth_prolongator)
    return AMG_ERR_ARG;
  const Level& L = H->L[level];
  cudaStream_t s = (cudaStream_t)stream;
  if (nnz) *nnz = L.p_nnz;
  if (w) *w = L.wp;
  if (rowptr)
    AMG_CUDA_TRY(cudaMemcpyAsync(rowptr, L.p_rp, sizeof(int64_t) * (L.n + 1),
                                 cudaMemcpyDeviceToDevice, s));
  if (col)
    AMG_CUDA_TRY(cudaMemcpyAsync(col, L.p_ci, sizeof(int32_t) * L.p_nnz,
                                 cudaMemcpyDeviceToDevice, s));
  if (val)
    AMG_CUDA_TRY(cudaMemcpyAsync(val, L.p_v, sizeof(double) * L.p_nnz, cudaMemcpyDeviceToDevice,
                                 s));
  return AMG_OK;
}

int amg_pairwise_match(const amg_csr* A, int32_t* mate, int* rounds, amg_stream_t stream) {
  int rc = check_csr(A);
  if (rc < 0) return rc;
  if (!mate) return AMG_ERR_ARG;
  Arena ar;
  rc = match_pairwise(ar, A->n, A->rowptr, A->col, A->val, mate, rounds, (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  ar.release_all();
  return rc;
}

}  // extern "C"
