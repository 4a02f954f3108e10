// Preconditioned conjugate gradient (Sec. 3; flexible CG with truncation 1)
// on the level-0 sliced-ELL matrix in FP64, preconditioned by the V-cycle.
//
//   r = b - A x;  z = B r;  p = z
//   repeat:  q = A p;  alpha = (r, z) / (p, q);  x += alpha p;  r -= alpha q
//            stop when ||r|| / ||b|| <= tol
//            z = B r;  beta = (r+, z+)/(r, z)  or  -(z+, q)/(p, q);  p = z + beta p
//
// Every dot product is fused into the kernel that produces its operands and
// reduced deterministically (per-block partials, summed in block order by the
// last block, which also computes alpha or beta on the device).  One
// iteration (V-cycle, p update, SpMV, update) can be replayed as a single
// captured CUDA graph; the host reads the scalars once per iteration for the
// convergence test.
#include <math.h>
#include <string.h>

#include "ring.cuh"
#include "sellk.cuh"

namespace amg {

struct InitEpi {
  PcgScalars* sc;
  __device__ void operator()(double (&t)[2]) const {
    sc->rr = t[0];
    sc->bb = t[1];
  }
};

struct TrueResEpi {
  PcgScalars* sc;
  __device__ void operator()(double (&t)[1]) const { sc->zq = t[0]; }
};

// r = b - A x with (r, r) and (b, b); mode 1 writes (r, r) to sc->zq only.
template <int TPR, int MODE>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_residual(SellView<double> A, const double* __restrict__ b, const double* __restrict__ x,
               double* __restrict__ r, Reduce red, PcgScalars* sc, float* __restrict__ r32) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double d[2] = {0.0, 0.0};
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < A.ngroups;
       sl += nw) {
    const double acc = sell_row<TPR, double>(A, sl, ln, [&](int j) { return __ldg(x + j); });
    const int64_t i = lane_row(A, sl, ln);
    if (i >= 0) {
      const double bi = b[i];
      const double ri = bi - acc;
      r[i] = ri;
      if (r32) r32[i] = (float)ri;
      d[0] += ri * ri;
      d[1] += bi * bi;
    }
  }
  if (MODE == 0) {
    grid_reduce<2>(d, red, InitEpi{sc});
  } else {
    double e[1] = {d[0]};
    grid_reduce<1>(e, red, TrueResEpi{sc});
  }
}

struct PqEpi {
  PcgScalars* sc;
  __device__ void operator()(double (&t)[1]) const {
    const double pq = t[0];
    sc->pq = pq;
    if (!(pq > 0.0)) {
      sc->status = isfinite(pq) ? AMG_ERR_BREAKDOWN : AMG_ERR_NAN;
      sc->pq_fail = 1;
    }
    sc->alpha = sc->rz / pq;
  }
};

// q = A p and (p, q); the last block sets alpha = (r, z) / (p, q).
template <int TPR>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_spmv_dot(SellView<double> A, const double* __restrict__ p, double* __restrict__ q,
               Reduce red, PcgScalars* sc) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double d[1] = {0.0};
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < A.ngroups;
       sl += nw) {
    const double acc = sell_row<TPR, double>(A, sl, ln, [&](int j) { return __ldg(p + j); });
    const int64_t i = lane_row(A, sl, ln);
    if (i >= 0) {
      q[i] = acc;
      d[0] += p[i] * acc;
    }
  }
  grid_reduce<1>(d, red, PqEpi{sc});
}

// k_spmv_dot on the shared-memory ring of ring.cuh (one system, one thread
// per row): the same row sums; (p, q) per thread over the warp's slices.
__global__ void __launch_bounds__(RING_THREADS, 4)
    k_spmv_dot_ring(SellView<double> A, const double* __restrict__ p, double* __restrict__ q,
                    Reduce red, PcgScalars* sc, RingGeom g, RingRows rows, int* fail) {
  extern __shared__ unsigned char ring_smem[];
  if (*(volatile int*)fail) return;  // the host resets the reduction ticket
  double d[1] = {0.0};
  RingWarp<double> ring(A, g, rows, ring_smem);
  ring.start();
  for (int64_t sl = ring.first; sl < A.nslices; sl += ring.nwt) {
    const int64_t i = sl * 32 + ring.lane;
    const bool has = i < A.n;
    const double pi = has ? __ldg(p + i) : 0.0;  // overlaps the wait
    if (!ring.wait()) {
      if (ring.lane == 0) ring_fail(fail, &sc->status);
      ring.drain();
      break;
    }
    const double acc =
        ring_row_sum<double>(ring, ring.width(), [&](int j) { return __ldg(p + j); });
    if (has) {
      q[i] = acc;
      d[0] += pi * acc;
    }
    ring.release();
  }
  grid_reduce<1>(d, red, PqEpi{sc});
}

struct RrEpi {
  PcgScalars* sc;
  __device__ void operator()(double (&t)[1]) const {
    sc->rr = t[0];
    if (!isfinite(t[0]) && sc->status == 0) sc->status = AMG_ERR_NAN;
  }
};

// x += alpha p; r -= alpha q; (r, r); r32 (if set) = (float) r for an FP32
// V-cycle, so it gathers 4-byte values without converting each one.
// Skipped after a breakdown.  x null: the x update is deferred to the next
// p update (k_p_update_x) or to the end of the solve (k_x_pending), which
// read p anyway; x_pending records that it is owed.
__global__ void k_cg_update(int64_t n, double* __restrict__ x, double* __restrict__ r,
                            const double* __restrict__ p, const double* __restrict__ q, Reduce red,
                            PcgScalars* sc, float* __restrict__ r32) {
  if (sc->status < 0) return;  // uniform across the grid: no block reduces
  const double alpha = sc->alpha;
  double d[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (x) x[i] = x[i] + alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    if (r32) r32[i] = (float)ri;
    d[0] += ri * ri;
  }
  if (!x && blockIdx.x == 0 && threadIdx.x == 0) sc->x_pending = 1;
  grid_reduce<1>(d, red, RrEpi{sc});
}

__global__ void k_p_update(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                           const PcgScalars* sc) {
  const double beta = sc->beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// The owed x += alpha p of the previous update (the loop only goes on after a
// complete one), then p = z + beta p: one pass over p for both.  The same
// expressions as k_cg_update and k_p_update, so the same bits.
__global__ void k_p_update_x(int64_t n, double* __restrict__ p, const double* __restrict__ z,
                             double* __restrict__ x, PcgScalars* sc) {
  const double alpha = sc->alpha, beta = sc->beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = p[i];
    x[i] = x[i] + alpha * pi;
    p[i] = z[i] + beta * pi;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->x_pending = 0;  // nobody else reads it here
}

// End of a solve: the x update still owed, if any.
__global__ void k_x_pending(int64_t n, double* __restrict__ x, const double* __restrict__ p,
                            const PcgScalars* sc) {
  if (!sc->x_pending) return;
  const double alpha = sc->alpha;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = x[i] + alpha * p[i];
}

// ------------------------------------------------------------------ driver

static int launch_residual(const amg_handle* H, int mode, const double* b, const double* x,
                           double* r, cudaStream_t s) {
  const Level& L = H->L[0];
  const int grid = sell_grid(sell_groups(L.A), H->num_sms);
  const SellView<double> v = view<double>(L.A, L.A.v64);
  if (mode == 0) {
    AMG_DISPATCH_TPR(sell_code(L.A), (k_residual<TPR, 0><<<grid, SELL_BLOCK, 0, s>>>(
                                  v, b, x, r, H->red, H->sc, H->r32)));
  } else {
    AMG_DISPATCH_TPR(sell_code(L.A), (k_residual<TPR, 1><<<grid, SELL_BLOCK, 0, s>>>(
                                  v, b, x, r, H->red, H->sc, nullptr)));
  }
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

static int launch_spmv_dot(const amg_handle* H, cudaStream_t s) {
  const Level& L = H->L[0];
  const int grid = sell_grid(sell_groups(L.A), H->num_sms);
  const SellView<double> v = view<double>(L.A, L.A.v64);
  if (H->opt.stream_ring && !H->batched) {
    RingGeom g = ring_plan(L.A, 8, ring_stages(H), RingRows());
    if (g.D) {
      AMG_TRY(ring_prepare((const void*)k_spmv_dot_ring, g, L.A.nslices, H->num_sms));
      k_spmv_dot_ring<<<g.grid, RING_THREADS, g.smem, s>>>(v, H->p, H->q, H->red, H->sc, g,
                                                           RingRows(), H->wait_fail);
      AMG_LAUNCH_CHECK();
      return AMG_OK;
    }
  }
  AMG_DISPATCH_TPR(sell_code(L.A),
                   (k_spmv_dot<TPR><<<grid, SELL_BLOCK, 0, s>>>(v, H->p, H->q, H->red, H->sc)));
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// defer: x += alpha p waits for the next p update (which reads p anyway),
// saving one pass over p per iteration; the solve then ends with
// k_x_pending.  Not with per-iteration histories of x.
static int launch_update(const amg_handle* H, double* x, bool defer, cudaStream_t s) {
  const int64_t n = H->L[0].n;
  k_cg_update<<<grid_for(n, 256, H->num_sms, 8), 256, 0, s>>>(
      n, defer ? nullptr : x, H->r, H->p, H->q, H->red, H->sc, H->r32);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

// One iteration after the first: z = B r (+ dots, beta), p = z + beta p
// (with the owed x update when deferring), q = A p (+ alpha), x/r update
// (+ (r, r)).
static int iteration_body(const amg_handle* H, double* x, int dots, bool defer, cudaStream_t s) {
  const int64_t n = H->L[0].n;
  AMG_TRY(vcycle_run(H, H->r, H->z, dots, H->q, s, nullptr, H->r32));
  if (defer)
    k_p_update_x<<<grid_for(n, 256, H->num_sms, 8), 256, 0, s>>>(n, H->p, H->z, x, H->sc);
  else
    k_p_update<<<grid_for(n, 256, H->num_sms, 8), 256, 0, s>>>(n, H->p, H->z, H->sc);
  AMG_LAUNCH_CHECK();
  AMG_TRY(launch_spmv_dot(H, s));
  AMG_TRY(launch_update(H, x, defer, s));
  return AMG_OK;
}

static int ensure_graph(amg_handle* H, double* x, int dots, int beta_form, bool defer) {
  if (H->graph && H->graph_x == x && H->graph_beta == beta_form &&
      H->graph_defer == (int)defer)
    return AMG_OK;
  if (H->graph) {
    cudaGraphExecDestroy(H->graph);
    H->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  AMG_CUDA_TRY(cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = iteration_body(H, x, dots, defer, H->cap_stream);
  cudaError_t e = cudaStreamEndCapture(H->cap_stream, &g);
  if (rc < 0) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  AMG_CUDA_TRY(e);
  e = cudaGraphInstantiate(&H->graph, g, 0);
  cudaGraphDestroy(g);
  AMG_CUDA_TRY(e);
  H->graph_x = x;
  H->graph_beta = beta_form;
  H->graph_defer = (int)defer;
  return AMG_OK;
}

// The stopping test of one iteration, on the device: the same decisions as
// the host loop in pcg_run (a failed (p, q) ends the solve without counting
// the step; otherwise count it, then stop on an error, on ||r||/||b|| <= tol
// or at maxit).  Sets the while-node condition: 1 = run another iteration.
__global__ void k_pcg_control(PcgScalars* sc, cudaGraphConditionalHandle h) {
  unsigned go = 0;
  if (!sc->pq_fail) {
    const int k = ++sc->iter;
    double bnorm = sqrt(sc->bb);
    if (bnorm == 0.0) bnorm = 1.0;
    const double rel = sqrt(sc->rr) / bnorm;
    go = (sc->status < 0 || rel <= sc->tol || k >= sc->maxit) ? 0u : 1u;
  }
  cudaGraphSetConditional(h, go);
}

int build_while_graph(cudaStream_t cs, const std::function<int(cudaStream_t)>& body,
                      const std::function<void(cudaStream_t, cudaGraphConditionalHandle)>& ctl,
                      cudaGraphExec_t* out) {
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaGraph_t g = nullptr;
  AMG_CUDA_TRY(cudaGraphCreate(&g, 0));
  int rc = AMG_OK;
  cudaGraphConditionalHandle h;
  cudaGraphNode_t first = nullptr, wnode = nullptr;
  size_t nn = 1;
  cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
  cudaGraph_t cap = nullptr;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, mode);
  if (e == cudaSuccess) {
    ctl(cs, h);
    e = cudaStreamEndCapture(cs, &cap);
  }
  if (e == cudaSuccess) e = cudaGraphGetNodes(g, &first, &nn);
  if (e == cudaSuccess && nn != 1) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) {
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&wnode, g, &first, nullptr, 1, &cp);
  }
  if (e == cudaSuccess)
    e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      mode);
  if (e == cudaSuccess) {
    rc = body(cs);
    if (rc == AMG_OK) ctl(cs, h);
    cudaGraph_t bcap = nullptr;
    e = cudaStreamEndCapture(cs, &bcap);
  }
  if (e == cudaSuccess && rc == AMG_OK) e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (rc < 0) return rc;
  if (e != cudaSuccess) {
    cudaGetLastError();
    *out = nullptr;
    return AMG_ERR_UNSUPPORTED;
  }
  return AMG_OK;
}

// The remaining iterations of a solve as one graph: the stopping test, then
// a conditional while node whose body is one iteration plus the test.  The
// host waits once per solve instead of once per iteration.
static int build_loop(amg_handle* H, double* x, int dots, cudaGraphExec_t* out) {
  PcgScalars* sc = H->sc;
  return build_while_graph(
      H->cap_stream, [&](cudaStream_t cs) { return iteration_body(H, x, dots, true, cs); },
      [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
        k_pcg_control<<<1, 1, 0, cs>>>(sc, h);
      },
      out);
}

// Loop graph for (x, beta form); AMG_ERR_UNSUPPORTED (once, remembered) if
// the runtime cannot build it, and the caller uses one graph per iteration.
static int ensure_loop(amg_handle* H, double* x, int dots, int beta_form) {
  if (H->loop_state < 0) return AMG_ERR_UNSUPPORTED;
  if (H->loop && H->loop_x == x && H->loop_beta == beta_form) return AMG_OK;
  if (H->loop) {
    cudaGraphExecDestroy(H->loop);
    H->loop = nullptr;
  }
  const int rc = build_loop(H, x, dots, &H->loop);
  if (rc == AMG_ERR_UNSUPPORTED) H->loop_state = -1;
  if (rc < 0) return rc;
  H->loop_state = 1;
  H->loop_x = x;
  H->loop_beta = beta_form;
  return AMG_OK;
}

static int read_scalars(amg_handle* H, cudaStream_t s) {
  AMG_CUDA_TRY(cudaMemcpyAsync(H->sc_host, H->sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  return AMG_OK;
}

int pcg_run(amg_handle* H, const double* b, double* x, const pcg_options* o, pcg_stats* st,
            cudaStream_t s) {
  const int64_t n = H->L[0].n;
  int beta_form = o->beta_form;
  if (beta_form == PCG_BETA_AUTO)
    beta_form = H->opt.precision == AMG_PREC_F32 ? PCG_BETA_FLEXIBLE : PCG_BETA_FR;
  const int dots = beta_form == PCG_BETA_FLEXIBLE ? 2 : 1;
  // one graph for the whole loop unless per-iteration histories are kept
  bool use_loop = false;
  if (o->use_graph == 1 && !o->res_history && !o->x_history) {
    const int rc = ensure_loop(H, x, dots, beta_form);
    if (rc < 0 && rc != AMG_ERR_UNSUPPORTED) return rc;
    use_loop = rc == AMG_OK;
  }
  // x updates are deferred (one pass over p saved per iteration) unless x is
  // recorded after every iteration
  const bool defer = !o->x_history;
  if (o->use_graph && !use_loop) AMG_TRY(ensure_graph(H, x, dots, beta_form, defer));

  PcgScalars init = {};
  init.beta_form = beta_form;
  init.tol = o->tol;
  init.maxit = o->maxit;
  *H->sc_host = init;
  AMG_CUDA_TRY(cudaMemcpyAsync(H->sc, H->sc_host, sizeof(PcgScalars), cudaMemcpyHostToDevice, s));
  AMG_CUDA_TRY(cudaEventRecord(H->ev0, s));
  AMG_TRY(launch_residual(H, 0, b, x, H->r, s));
  AMG_TRY(read_scalars(H, s));
  double bnorm = sqrt(H->sc_host->bb);
  if (bnorm == 0.0) bnorm = 1.0;
  double relres = sqrt(H->sc_host->rr) / bnorm;
  if (o->res_history) o->res_history[0] = relres;
  if (o->x_history)
    AMG_CUDA_TRY(cudaMemcpyAsync(o->x_history, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  int status = AMG_NOT_CONVERGED;
  int k = 0;
  if (relres <= o->tol) {
    status = AMG_OK;
  } else if (o->maxit > 0) {
    AMG_TRY(vcycle_run(H, H->r, H->z, dots, H->q, s, nullptr, H->r32));
    AMG_CUDA_TRY(cudaMemcpyAsync(H->p, H->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    AMG_TRY(launch_spmv_dot(H, s));
    AMG_TRY(launch_update(H, x, defer, s));
    if (use_loop) {
      AMG_CUDA_TRY(cudaGraphLaunch(H->loop, s));
      AMG_TRY(read_scalars(H, s));
      const PcgScalars& S = *H->sc_host;
      k = S.iter;
      relres = sqrt(S.rr) / bnorm;  // rr is left unchanged by a failed step
      if (S.pq_fail || S.status < 0)
        status = S.status;
      else if (relres <= o->tol)
        status = AMG_OK;
    }
    for (; !use_loop;) {
      AMG_TRY(read_scalars(H, s));
      const int dstat = H->sc_host->status;
      if (H->sc_host->pq_fail) {  // x and r were not updated in this step
        status = dstat;
        break;
      }
      ++k;
      relres = sqrt(H->sc_host->rr) / bnorm;
      if (o->res_history) o->res_history[k] = relres;
      if (o->x_history)
        AMG_CUDA_TRY(cudaMemcpyAsync(o->x_history + (int64_t)k * n, x, sizeof(double) * n,
                                     cudaMemcpyDeviceToDevice, s));
      if (dstat < 0) {
        status = dstat;
        break;
      }
      if (relres <= o->tol) {
        status = AMG_OK;
        break;
      }
      if (k >= o->maxit) break;
      if (o->use_graph) {
        AMG_CUDA_TRY(cudaGraphLaunch(H->graph, s));
      } else {
        AMG_TRY(iteration_body(H, x, dots, defer, s));
      }
    }
    if (defer) {
      k_x_pending<<<grid_for(n, 256, H->num_sms, 8), 256, 0, s>>>(n, x, H->p, H->sc);
      AMG_LAUNCH_CHECK();
    }
  }
  AMG_CUDA_TRY(cudaEventRecord(H->ev1, s));
  // true residual ||b - A x|| / ||b|| (outside the timed region)
  AMG_TRY(launch_residual(H, 1, b, x, H->z, s));
  AMG_TRY(read_scalars(H, s));
  const int tc = tail_check(H, s);
  if (tc < 0) status = tc;
  float ms = 0.f;
  AMG_CUDA_TRY(cudaEventElapsedTime(&ms, H->ev0, H->ev1));
  if (st) {
    st->iterations = k;
    st->status = status;
    st->rel_residual = relres;
    st->true_rel_residual = sqrt(H->sc_host->zq) / bnorm;
    st->solve_ms = ms;
  }
  return status;
}

}  // namespace amg
