// Batched PCG over many independent SPD systems (pcg_solve_batch).
//
// The systems are concatenated into one block-diagonal matrix.  Matching and
// the Galerkin product never couple two blocks, so the hierarchy built from
// it is block diagonal too and every V-cycle kernel applies each system's own
// V-cycle (one launch per stage for all systems).  Every level is sliced so
// that no slice straddles two systems: the slices form a work list of
// (system, slice) tiles.  The PCG kernels below walk the level-0 tiles, write
// partial sums, and a segmented reduction turns those into the
// per-system scalars (alpha, beta, residual norm) and convergence flags on the
// device.  Partial sums are per chunk of up to BATCH_CHUNK slices of one
// system (a warp walks a chunk and reduces once at its end).  Converged
// systems are frozen: their tiles are skipped in the SpMV and vector updates.  One iteration for all systems replays as one CUDA
// graph; the host reads only the number of systems still iterating.
#include <math.h>

#include <algorithm>

#include "sellk.cuh"

namespace amg {

enum { SEG_INIT = 0, SEG_RZ_FIRST = 1, SEG_PQ = 2, SEG_RR = 3, SEG_RZ = 4, SEG_TRUE = 5 };

// The kernels below walk the level-0 chunks (Batch): warp w takes chunks
// w, w + W, ...; a chunk is consecutive slices of one system.
#define AMG_BATCH_CHUNKS(c, s0, s1)                                                     \
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks;  \
       c += ((int64_t)gridDim.x * blockDim.x) >> 5)                                     \
    for (int64_t s0 = chunk_off[c], s1 = chunk_off[c + 1], once_ = 1; once_; once_ = 0)

// r = b - A x with per-chunk (r, r) and (b, b).
template <int TPR>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_b_residual(SellView<double> A, int64_t nchunks, const int64_t* __restrict__ chunk_off,
                 const double* __restrict__ b, const double* __restrict__ x,
                 double* __restrict__ r, double* __restrict__ part, float* __restrict__ r32) {
  const Lanes<TPR> ln;
  AMG_BATCH_CHUNKS(c, s0, s1) {
    double d0 = 0.0, d1 = 0.0;
    for (int64_t sl = s0; sl < s1; ++sl) {
      const double acc = sell_row<TPR, double>(A, sl, ln, [&](int j) { return __ldg(x + j); });
      const int64_t i = lane_row(A, sl, ln);
      if (i >= 0) {
        const double ri = b[i] - acc;
        r[i] = ri;
        if (r32) r32[i] = (float)ri;
        d0 += ri * ri;
        d1 += b[i] * b[i];
      }
    }
    d0 = warp_sum(d0);
    d1 = warp_sum(d1);
    if ((threadIdx.x & 31) == 0) {
      part[2 * c] = d0;
      part[2 * c + 1] = d1;
    }
  }
}

// q = A p with per-chunk (p, q); chunks of converged systems are skipped.
template <int TPR>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_b_spmv_dot(SellView<double> A, int64_t nchunks, const int64_t* __restrict__ chunk_off,
                 const double* __restrict__ p, double* __restrict__ q,
                 double* __restrict__ part, const Scal* __restrict__ sc) {
  const Lanes<TPR> ln;
  AMG_BATCH_CHUNKS(c, s0, s1) {
    if (!sc[A.sys[s0]].active) continue;  // warp-uniform: one system per chunk
    double d = 0.0;
    for (int64_t sl = s0; sl < s1; ++sl) {
      const double acc = sell_row<TPR, double>(A, sl, ln, [&](int j) { return __ldg(p + j); });
      const int64_t i = lane_row(A, sl, ln);
      if (i >= 0) {
        q[i] = acc;
        d += p[i] * acc;
      }
    }
    d = warp_sum(d);
    if ((threadIdx.x & 31) == 0) part[2 * c] = d;
  }
}

// x += alpha_k p; r -= alpha_k q; per-chunk (r, r); r32 (if set) = (float) r.
__global__ void k_b_update(SellView<double> A, int64_t nchunks,
                           const int64_t* __restrict__ chunk_off, double* __restrict__ x,
                           double* __restrict__ r, const double* __restrict__ p,
                           const double* __restrict__ q, double* __restrict__ part,
                           const Scal* __restrict__ sc, float* __restrict__ r32) {
  const int lane = threadIdx.x & 31;
  AMG_BATCH_CHUNKS(c, s0, s1) {
    const Scal& S = sc[A.sys[s0]];
    if (!S.active) continue;
    const double alpha = S.alpha;
    double d = 0.0;
    // the chunk's rows are contiguous: first row of its first slice to one past
    // the last row of its last
    for (int64_t i = A.rbeg(s0, 32) + lane; i < A.rend(s1 - 1, 32); i += 32) {
      x[i] = x[i] + alpha * p[i];
      const double ri = r[i] - alpha * q[i];
      r[i] = ri;
      if (r32) r32[i] = (float)ri;
      d += ri * ri;
    }
    d = warp_sum(d);
    if (lane == 0) part[2 * c] = d;
  }
}

// p = z + beta_k p on the tiles of systems still iterating.
__global__ void k_b_p_update(SellView<double> A, double* __restrict__ p,
                             const double* __restrict__ z, const Scal* __restrict__ sc) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < A.nslices;
       sl += nw) {
    const Scal& S = sc[A.sys[sl]];
    if (!S.active) continue;
    const double beta = S.beta;
    for (int64_t i = A.rbeg(sl, 32) + lane; i < A.rend(sl, 32); i += 32) p[i] = z[i] + beta * p[i];
  }
}

// One CUDA block per system: each thread sums a fixed stride of its chunks'
// partials, the block adds them by a fixed tree, and thread 0 updates that
// system's scalars (deterministic run to run).
template <int MODE>
__global__ void k_b_seg(int nsys, const int64_t* __restrict__ sys_chunk,
                        const double* __restrict__ part, Scal* sc, double tol, int maxit,
                        int beta_form, int* nactive, int* active) {
  for (int k = blockIdx.x; k < nsys; k += gridDim.x) {
    double t[2] = {0.0, 0.0};
    for (int64_t c = sys_chunk[k] + threadIdx.x; c < sys_chunk[k + 1]; c += blockDim.x) {
      t[0] += part[2 * c];
      t[1] += part[2 * c + 1];
    }
    block_sum<2>(t);
    const double t0 = t[0], t1 = t[1];
    __syncthreads();  // the block's shared scratch is reused by the next system
    if (threadIdx.x != 0) continue;
    Scal& S = sc[k];
    if (MODE == SEG_INIT) {
      S.rr = t0;
      S.bb = t1;
      S.iters = 0;
      S.status = AMG_NOT_CONVERGED;
      S.pq_fail = 0;
      const double bn = t1 > 0.0 ? sqrt(t1) : 1.0;
      S.active = (sqrt(t0) / bn > tol && maxit > 0) ? 1 : 0;
      if (sqrt(t0) / bn <= tol) S.status = AMG_OK;
      if (S.active) atomicAdd(nactive, 1);
    } else if (MODE == SEG_RZ_FIRST) {
      S.rz = t0;
    } else if (MODE == SEG_TRUE) {
      S.tr = t0;
    } else if (S.active) {
      if (MODE == SEG_PQ) {
        S.pq = t0;
        if (!(t0 > 0.0)) {
          S.status = isfinite(t0) ? AMG_ERR_BREAKDOWN : AMG_ERR_NAN;
          S.pq_fail = 1;
          S.active = 0;
        }
        S.alpha = S.rz / t0;
      } else if (MODE == SEG_RR) {
        S.rr = t0;
        S.iters += 1;
        const double bn = S.bb > 0.0 ? sqrt(S.bb) : 1.0;
        const double rel = sqrt(t0) / bn;
        if (!isfinite(t0)) {
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
      } else if (MODE == SEG_RZ) {
        S.beta = beta_form == PCG_BETA_FLEXIBLE ? -t1 / S.pq : t0 / S.rz;
        S.zq = t1;
        S.rz = t0;
        if (!isfinite(t0)) {
          S.status = AMG_ERR_NAN;
          S.active = 0;
        }
      }
    }
    active[k] = S.active;
  }
}

// ------------------------------------------------------------------ driver

struct BatchRun {
  const amg_handle* H;
  double tol;
  int maxit, beta_form, dots;
};

template <int MODE>
static int seg(const BatchRun& R, cudaStream_t s) {
  const Batch& B = R.H->batch;
  const int grid = std::max(1, std::min(B.nsys, R.H->num_sms * 8));
  k_b_seg<MODE><<<grid, 256, 0, s>>>(B.nsys, B.sys_chunk, B.part, B.sc, R.tol, R.maxit,
                                     R.beta_form, B.nactive, B.active);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

static SellView<double> a0(const amg_handle* H) { return view<double>(H->L[0].A, H->L[0].A.v64); }

// Grid of the chunk kernels: one warp per chunk, at most one full wave.
static int chunk_grid(const amg_handle* H) { return sell_grid(H->batch.nchunks, H->num_sms); }

static int b_residual(const BatchRun& R, const double* b, const double* x, double* r,
                      float* r32, cudaStream_t s) {
  const Level& L = R.H->L[0];
  const Batch& B = R.H->batch;
  AMG_DISPATCH_TPR(sell_code(L.A), (k_b_residual<TPR><<<chunk_grid(R.H), SELL_BLOCK, 0, s>>>(
                                a0(R.H), B.nchunks, B.chunk_off, b, x, r, B.part, r32)));
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

static int b_spmv_dot(const amg_handle* H, cudaStream_t s) {
  const Batch& B = H->batch;
  AMG_DISPATCH_TPR(sell_code(H->L[0].A),
                   (k_b_spmv_dot<TPR><<<chunk_grid(H), SELL_BLOCK, 0, s>>>(
                       a0(H), B.nchunks, B.chunk_off, H->p, H->q, B.part, B.sc)));
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

static int b_update(const amg_handle* H, double* x, cudaStream_t s) {
  const Batch& B = H->batch;
  k_b_update<<<chunk_grid(H), SELL_BLOCK, 0, s>>>(a0(H), B.nchunks, B.chunk_off, x, H->r, H->p,
                                                  H->q, B.part, B.sc, H->r32);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// One iteration after the first: z = B r, beta, p, q = A p, alpha, x/r, convergence.
static int b_body(const BatchRun& R, double* x, cudaStream_t s) {
  const amg_handle* H = R.H;
  const Level& L = H->L[0];
  const int grid = sell_grid(L.A.nslices, H->num_sms);
  AMG_TRY(vcycle_run(H, H->r, H->z, R.dots, H->q, s, H->batch.part, H->r32));
  AMG_TRY(seg<SEG_RZ>(R, s));
  k_b_p_update<<<grid, SELL_BLOCK, 0, s>>>(a0(H), H->p, H->z, H->batch.sc);
  AMG_LAUNCH_CHECK();
  AMG_TRY(b_spmv_dot(H, s));
  AMG_TRY(seg<SEG_PQ>(R, s));
  AMG_TRY(b_update(H, x, s));
  AMG_CUDA_TRY(cudaMemsetAsync(H->batch.nactive, 0, sizeof(int), s));
  AMG_TRY(seg<SEG_RR>(R, s));
  return AMG_OK;
}

// Stopping test of the batched loop graph, the host loop's test on the
// device: another iteration while a system is active and fewer than maxit
// iterations were taken (ctl[0] counts them, ctl[1] is maxit).
__global__ void k_b_control(const int* nactive, int* ctl, cudaGraphConditionalHandle h) {
  const int k = ctl[0];
  const unsigned go = (*nactive > 0 && k < ctl[1]) ? 1u : 0u;
  if (go) ctl[0] = k + 1;
  cudaGraphSetConditional(h, go);
}

// Per-iteration graph (host-driven loop), keyed on everything it bakes in.
static int ensure_bgraph(amg_handle* H, const BatchRun& R, double* x) {
  if (H->bgraph && H->bgraph_x == x && H->bgraph_beta == R.beta_form &&
      H->bgraph_tol == R.tol && H->bgraph_maxit == R.maxit)
    return AMG_OK;
  if (H->bgraph) {
    cudaGraphExecDestroy(H->bgraph);
    H->bgraph = nullptr;
  }
  cudaGraph_t g = nullptr;
  AMG_CUDA_TRY(cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = b_body(R, x, H->cap_stream);
  cudaError_t e = cudaStreamEndCapture(H->cap_stream, &g);
  if (rc < 0) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  AMG_CUDA_TRY(e);
  e = cudaGraphInstantiate(&H->bgraph, g, 0);
  cudaGraphDestroy(g);
  AMG_CUDA_TRY(e);
  H->bgraph_x = x;
  H->bgraph_beta = R.beta_form;
  H->bgraph_tol = R.tol;
  H->bgraph_maxit = R.maxit;
  return AMG_OK;
}

// All remaining iterations as one graph; AMG_ERR_UNSUPPORTED (remembered)
// when the runtime cannot build it.
static int ensure_bloop(amg_handle* H, const BatchRun& R, double* x) {
  if (H->bloop_state < 0) return AMG_ERR_UNSUPPORTED;
  if (H->bloop && H->bloop_x == x && H->bloop_beta == R.beta_form && H->bloop_tol == R.tol &&
      H->bloop_maxit == R.maxit)
    return AMG_OK;
  if (H->bloop) {
    cudaGraphExecDestroy(H->bloop);
    H->bloop = nullptr;
  }
  const Batch& B = H->batch;
  const int rc = build_while_graph(
      H->cap_stream, [&](cudaStream_t cs) { return b_body(R, x, cs); },
      [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
        k_b_control<<<1, 1, 0, cs>>>(B.nactive, B.loop_ctl, h);
      },
      &H->bloop);
  if (rc == AMG_ERR_UNSUPPORTED) H->bloop_state = -1;
  if (rc < 0) return rc;
  H->bloop_state = 1;
  H->bloop_x = x;
  H->bloop_beta = R.beta_form;
  H->bloop_tol = R.tol;
  H->bloop_maxit = R.maxit;
  return AMG_OK;
}

static int read_nactive(const amg_handle* H, int* h, cudaStream_t s) {
  AMG_CUDA_TRY(cudaMemcpyAsync(h, H->batch.nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  return AMG_OK;
}

int pcg_batch_run(amg_handle* H, const double* b, double* x, const pcg_options* o, pcg_stats* st,
                  cudaStream_t s) {
  const int64_t n = H->L[0].n;
  int beta_form = o->beta_form;
  if (beta_form == PCG_BETA_AUTO)
    beta_form = H->opt.precision == AMG_PREC_F32 ? PCG_BETA_FLEXIBLE : PCG_BETA_FR;
  BatchRun R{H, o->tol, o->maxit, beta_form, beta_form == PCG_BETA_FLEXIBLE ? 2 : 1};
  const Batch& B = H->batch;
  const int grid = sell_grid(H->L[0].A.nslices, H->num_sms);
  bool use_loop = false;
  if (o->use_graph == 1) {
    const int rc = ensure_bloop(H, R, x);
    if (rc < 0 && rc != AMG_ERR_UNSUPPORTED) return rc;
    use_loop = rc == AMG_OK;
  }
  if (o->use_graph && !use_loop) AMG_TRY(ensure_bgraph(H, R, x));
  AMG_CUDA_TRY(cudaEventRecord(H->ev0, s));
  AMG_TRY(b_residual(R, b, x, H->r, H->r32, s));
  AMG_CUDA_TRY(cudaMemsetAsync(B.nactive, 0, sizeof(int), s));
  AMG_TRY(seg<SEG_INIT>(R, s));
  int act = 0;
  AMG_TRY(read_nactive(H, &act, s));
  int k = 0;
  if (act > 0) {
    AMG_TRY(vcycle_run(H, H->r, H->z, R.dots, H->q, s, B.part, H->r32));
    AMG_TRY(seg<SEG_RZ_FIRST>(R, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(H->p, H->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    AMG_TRY(b_spmv_dot(H, s));
    AMG_TRY(seg<SEG_PQ>(R, s));
    AMG_TRY(b_update(H, x, s));
    AMG_CUDA_TRY(cudaMemsetAsync(B.nactive, 0, sizeof(int), s));
    AMG_TRY(seg<SEG_RR>(R, s));
    k = 1;
    if (use_loop) {
      const int ctl[2] = {1, o->maxit};
      AMG_CUDA_TRY(cudaMemcpyAsync(B.loop_ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, s));
      AMG_CUDA_TRY(cudaGraphLaunch(H->bloop, s));
    }
    for (; !use_loop;) {
      AMG_TRY(read_nactive(H, &act, s));
      if (act == 0 || k >= o->maxit) break;
      if (o->use_graph)
        AMG_CUDA_TRY(cudaGraphLaunch(H->bgraph, s));
      else
        AMG_TRY(b_body(R, x, s));
      ++k;
    }
  }
  AMG_CUDA_TRY(cudaEventRecord(H->ev1, s));
  AMG_TRY(b_residual(R, b, x, H->z, nullptr, s));
  AMG_TRY(seg<SEG_TRUE>(R, s));
  AMG_CUDA_TRY(cudaMemcpyAsync(B.sc_host, B.sc, sizeof(Scal) * B.nsys, cudaMemcpyDeviceToHost, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  float ms = 0.f;
  AMG_CUDA_TRY(cudaEventElapsedTime(&ms, H->ev0, H->ev1));
  int worst = AMG_OK;
  for (int i = 0; i < B.nsys; ++i) {
    const Scal& S = B.sc_host[i];
    const double bn = S.bb > 0.0 ? sqrt(S.bb) : 1.0;
    if (st) {
      st[i].iterations = S.iters;
      st[i].status = S.status;
      st[i].rel_residual = sqrt(S.rr) / bn;
      st[i].true_rel_residual = sqrt(S.tr) / bn;
      st[i].solve_ms = ms;
    }
    if (S.status < 0 && (worst >= 0 || S.status < worst)) worst = S.status;
    if (S.status == AMG_NOT_CONVERGED && worst == AMG_OK) worst = AMG_NOT_CONVERGED;
  }
  const int tc = tail_check(H, s);
  return tc < 0 ? tc : worst;
}

// Batch bookkeeping after the hierarchy exists: tile ranges per system.
int batch_init(amg_handle* H, cudaStream_t s) {
  Batch& B = H->batch;
  const Level& L = H->L[0];
  B.nsys = H->nsys;
  B.nslices = L.A.nslices;
  std::vector<int64_t> off(B.nsys + 1, 0);
  for (int k = 0; k < B.nsys; ++k) {
    const int64_t rows = L.sys_off[k + 1] - L.sys_off[k];
    off[k + 1] = off[k] + (rows + L.A.C - 1) / L.A.C;
  }
  if (off.back() != B.nslices) return AMG_ERR_DEVICE_CHECK;
  // chunks of at most BATCH_CHUNK slices, never across two systems
  std::vector<int64_t> coff, sch(B.nsys + 1, 0);
  for (int k = 0; k < B.nsys; ++k) {
    sch[k] = (int64_t)coff.size();
    for (int64_t sl = off[k]; sl < off[k + 1]; sl += BATCH_CHUNK) coff.push_back(sl);
  }
  sch[B.nsys] = (int64_t)coff.size();
  B.nchunks = (int64_t)coff.size();
  coff.push_back(B.nslices);
  Arena& ar = H->arena;
  AMG_TRY(ar.alloc_n(&B.slice_off, B.nsys + 1));
  AMG_TRY(ar.alloc_n(&B.chunk_off, B.nchunks + 1));
  AMG_TRY(ar.alloc_n(&B.sys_chunk, B.nsys + 1));
  AMG_TRY(ar.alloc_n(&B.part, 2 * B.nchunks));
  AMG_TRY(ar.alloc_n(&B.sc, B.nsys));
  AMG_TRY(ar.alloc_n(&B.nactive, 1));
  AMG_TRY(ar.alloc_n(&B.loop_ctl, 2));
  AMG_TRY(ar.alloc_n(&B.active, B.nsys));
  AMG_CUDA_TRY(cudaMallocHost((void**)&B.sc_host, sizeof(Scal) * B.nsys));
  AMG_CUDA_TRY(cudaMemcpyAsync(B.slice_off, off.data(), sizeof(int64_t) * off.size(),
                               cudaMemcpyHostToDevice, s));
  AMG_CUDA_TRY(cudaMemcpyAsync(B.chunk_off, coff.data(), sizeof(int64_t) * coff.size(),
                               cudaMemcpyHostToDevice, s));
  AMG_CUDA_TRY(cudaMemcpyAsync(B.sys_chunk, sch.data(), sizeof(int64_t) * sch.size(),
                               cudaMemcpyHostToDevice, s));
  AMG_CUDA_TRY(cudaMemsetAsync(B.part, 0, sizeof(double) * 2 * B.nchunks, s));
  AMG_CUDA_TRY(cudaMemsetAsync(B.sc, 0, sizeof(Scal) * B.nsys, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  return AMG_OK;
}

// ------------------------------------------------------------------ concatenation

__global__ void k_cat_rowptr(int64_t n, const int64_t* rp, int64_t nnz_off, int64_t* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = rp[i] - rp[0] + nnz_off;
}

__global__ void k_cat_col(int64_t nnz, const int32_t* col, int64_t row_off, int32_t* out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (int32_t)(col[e] + row_off);
}

int concat_systems(Arena& ar, int nsys, const amg_csr* A, amg_csr* cat, int64_t** rp,
                   int32_t** ci, double** va, std::vector<int64_t>& off, int num_sms,
                   cudaStream_t s) {
  int64_t n = 0, nnz = 0;
  off.assign(nsys + 1, 0);
  for (int k = 0; k < nsys; ++k) {
    off[k + 1] = off[k] + A[k].n;
    n += A[k].n;
    nnz += A[k].nnz;
  }
  if (n > (int64_t)0x7fffffff) return AMG_ERR_UNSUPPORTED;
  AMG_TRY(ar.alloc_n(rp, n + 1));
  AMG_TRY(ar.alloc_n(ci, nnz));
  AMG_TRY(ar.alloc_n(va, nnz));
  int64_t e0 = 0;
  for (int k = 0; k < nsys; ++k) {
    const amg_csr& a = A[k];
    k_cat_rowptr<<<grid_for(a.n + 1, 256, num_sms, 4), 256, 0, s>>>(a.n, a.rowptr, e0,
                                                                      *rp + off[k]);
    AMG_LAUNCH_CHECK();
    int64_t base = 0;  // entries of system k start at its rowptr[0]
    AMG_CUDA_TRY(cudaMemcpyAsync(&base, a.rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    k_cat_col<<<grid_for(a.nnz, 256, num_sms, 4), 256, 0, s>>>(a.nnz, a.col + base, off[k],
                                                                *ci + e0);
    AMG_LAUNCH_CHECK();
    AMG_CUDA_TRY(cudaMemcpyAsync(*va + e0, a.val + base, sizeof(double) * a.nnz,
                                 cudaMemcpyDeviceToDevice, s));
    e0 += a.nnz;
  }
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  cat->n = n;
  cat->nnz = nnz;
  cat->rowptr = *rp;
  cat->col = *ci;
  cat->val = *va;
  return AMG_OK;
}

}  // namespace amg
