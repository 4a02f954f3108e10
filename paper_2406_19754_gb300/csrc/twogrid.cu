// Two-grid error-reduction loss of the level-0 smoother weights and its
// gradient, the training signal for the learned smoother.
//
//   L = mean_j log(||E^K e0_j||_A / ||e0_j||_A) / K,
//   E = S (I - P A_c^-1 P^T A) S,   S = I - diag(s) A,  s_i = omega_i / d_i,
//
// with P the level-0 aggregate map and A_c the level-1 matrix (Sec. 2.3:
// Eq. amg with two levels, l1-Jacobi smoother).  A_c^-1 is applied by PCG
// preconditioned with the hierarchy of levels >= 1 (a second handle) to a
// relative residual of 1e-12, or exactly by Cholesky when level 1 is the
// coarsest.  The gradient comes from the adjoint pass: S and the coarse
// correction are linear, S^T = I - A diag(s) and
// (I - P A_c^-1 P^T A)^T = I - A P A_c^-1 P^T, run in reverse order over the
// stored forward states, with d(S x)_i / d s_i = -(A x)_i.  All FP64.
#include <math.h>

#include <type_traits>
#include <vector>

#include "sellk.cuh"

namespace amg {

template <int TPR>
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_tg_smooth(SellView<double> A, const double* __restrict__ s, const double* __restrict__ x,
                double* __restrict__ out, double* __restrict__ Ax) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < A.ngroups;
       sl += nw) {
    const double acc = sell_row<TPR, double>(A, sl, ln, [&](int j) { return __ldg(x + j); });
    const int64_t i = lane_row(A, sl, ln);
    if (i >= 0) {
      Ax[i] = acc;
      out[i] = x[i] - s[i] * acc;
    }
  }
}

enum { TG_PROLONG_SUB = 0, TG_PROLONG = 1, TG_SCALE_S = 2, TG_SUB = 3, TG_SBAR = 4,
       TG_SCALE = 5, TG_DOMEGA = 6 };

// Elementwise steps of the forward and adjoint passes.
template <int OP>
__global__ void k_tg_vec(int64_t n, const double* __restrict__ x, const double* __restrict__ w,
                         const int32_t* __restrict__ agg, const double* __restrict__ s,
                         double c, double* __restrict__ out, float* __restrict__ outf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (OP == TG_PROLONG_SUB) out[i] = x[i] - w[agg[i]];  // x - P y
    if (OP == TG_PROLONG) out[i] = w[agg[i]];              // P y
    if (OP == TG_SCALE_S) out[i] = s[i] * x[i];            // diag(s) x
    if (OP == TG_SUB) out[i] = x[i] - w[i];
    if (OP == TG_SBAR) out[i] = out[i] - x[i] * w[i];      // sbar -= u o w
    if (OP == TG_SCALE) out[i] = c * x[i];
    if (OP == TG_DOMEGA) outf[i] = (float)(x[i] / w[i]);   // d L / d omega = sbar / d
  }
}

// g = P^T x: sum over each aggregate's members (ascending).
__global__ void k_tg_restrict(int64_t nc, int stride, const int32_t* __restrict__ members,
                              const double* __restrict__ x, double* __restrict__ g) {
  for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < nc;
       I += (int64_t)gridDim.x * blockDim.x) {
    const int32_t* m = members + I * stride;
    double acc = x[m[0]];
    for (int k = 1; k < stride && m[k] >= 0; ++k) acc = acc + x[m[k]];
    g[I] = acc;
  }
}

struct DotEpi {
  double* dst;
  __device__ void operator()(double (&t)[1]) const { *dst = t[0]; }
};

__global__ void k_tg_dot(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                         Reduce red, double* dst) {
  double d[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d[0] += x[i] * y[i];
  grid_reduce<1>(d, red, DotEpi{dst});
}

struct TgWs {
  int64_t n = 0, nc = 0;
  int K = 0;
  double *e = nullptr, *a = nullptr, *c = nullptr, *t = nullptr, *t2 = nullptr, *sbar = nullptr;
  double *eb = nullptr, *cb = nullptr, *ab = nullptr;
  double *g = nullptr, *y = nullptr, *dots = nullptr;
  std::vector<double*> Ae, Ac;
  double* dots_host = nullptr;  // pinned
};

}  // namespace amg

struct amg_tg {
  amg_handle* inner = nullptr;  // PCG-AMG on level 1
  amg::TgWs w;
};

namespace amg {

void tg_free(amg_handle* H) {
  amg_tg* T = (amg_tg*)H->tg;
  if (!T) return;
  if (T->inner) amg_destroy(T->inner);
  if (T->w.dots_host) cudaFreeHost(T->w.dots_host);
  delete T;
  H->tg = nullptr;
}

static int tg_prepare(amg_handle* H, int K, cudaStream_t s, amg_tg** out) {
  amg_tg* T = (amg_tg*)H->tg;
  if (T && T->w.K >= K) {
    *out = T;
    return AMG_OK;
  }
  Arena& ar = H->arena;
  if (!T) {
    T = new amg_tg();
    H->tg = T;
    const Level& L1 = H->L[1];
    amg_csr A1{L1.n, L1.nnz, L1.rowptr, L1.col, L1.val};
    amg_options o = H->opt;
    o.precision = AMG_PREC_F64;
    o.autotune = 0;
    AMG_TRY(amg_setup(&A1, &o, (amg_stream_t)s, &T->inner));
    const int64_t n = H->L[0].n, nc = L1.n;
    TgWs& w = T->w;
    w.n = n;
    w.nc = nc;
    for (double** p : {&w.e, &w.a, &w.c, &w.t, &w.t2, &w.sbar, &w.eb, &w.cb, &w.ab})
      AMG_TRY(ar.alloc_n(p, n));
    AMG_TRY(ar.alloc_n(&w.g, nc));
    AMG_TRY(ar.alloc_n(&w.y, nc));
    AMG_TRY(ar.alloc_n(&w.dots, 2));
    AMG_CUDA_TRY(cudaMallocHost((void**)&w.dots_host, 2 * sizeof(double)));
  }
  TgWs& w = T->w;
  while ((int)w.Ae.size() < K) {
    double *p = nullptr, *q = nullptr;
    AMG_TRY(ar.alloc_n(&p, w.n));
    AMG_TRY(ar.alloc_n(&q, w.n));
    w.Ae.push_back(p);
    w.Ac.push_back(q);
  }
  w.K = K;
  *out = T;
  return AMG_OK;
}

int twogrid_loss(amg_handle* H, int nsamples, int K, const double* e0, double* loss,
                 float* domega, cudaStream_t s) {
  if (H->L.size() < 2 || H->batched) return AMG_ERR_UNSUPPORTED;
  amg_tg* T = nullptr;
  AMG_TRY(tg_prepare(H, K, s, &T));
  TgWs& w = T->w;
  const Level& L0 = H->L[0];
  const int64_t n = w.n;
  const SellView<double> A = view<double>(L0.A, L0.A.v64);
  const int gs = sell_grid(sell_groups(L0.A), H->num_sms);
  const int gv = grid_for(n, 256, H->num_sms, 8);
  const double* sv = L0.s64;
  pcg_options po;
  pcg_default_options(&po);
  po.tol = 1e-12;
  po.maxit = 1000;
  po.beta_form = PCG_BETA_FR;
  auto spmv = [&](const double* x, double* y) {
    return sell_spmv64(L0.A, 1.0, x, 0.0, y, H->num_sms, s);
  };
  auto smooth = [&](const double* x, double* o, double* Ax) -> int {
    AMG_DISPATCH_TPR(sell_code(L0.A),
                     (k_tg_smooth<TPR><<<gs, SELL_BLOCK, 0, s>>>(A, sv, x, o, Ax)));
    AMG_LAUNCH_CHECK();
    return AMG_OK;
  };
  auto csolve = [&]() -> int {  // y = A_c^-1 g
    AMG_CUDA_TRY(cudaMemsetAsync(w.y, 0, sizeof(double) * w.nc, s));
    int rc = pcg_solve(T->inner, w.g, w.y, &po, nullptr, (amg_stream_t)s);
    return rc == AMG_NOT_CONVERGED ? AMG_OK : rc;  // 1e-12 is a target, not a requirement
  };
  auto restrict_ = [&](const double* x) -> int {  // g = P^T x
    k_tg_restrict<<<grid_for(L0.nc, 256, H->num_sms, 8), 256, 0, s>>>(L0.nc, L0.stride,
                                                                      L0.members, x, w.g);
    AMG_LAUNCH_CHECK();
    return AMG_OK;
  };
  auto vec = [&](auto op, const double* x, const double* y2, double c, double* o) -> int {
    k_tg_vec<decltype(op)::value><<<gv, 256, 0, s>>>(n, x, y2, L0.agg, sv, c, o, nullptr);
    AMG_LAUNCH_CHECK();
    return AMG_OK;
  };
  auto dot = [&](const double* x, const double* y2, int slot) -> int {
    k_tg_dot<<<gv, 256, 0, s>>>(n, x, y2, H->red, w.dots + slot);
    AMG_LAUNCH_CHECK();
    return AMG_OK;
  };
  using PS = std::integral_constant<int, TG_PROLONG_SUB>;
  using PR = std::integral_constant<int, TG_PROLONG>;
  using SS = std::integral_constant<int, TG_SCALE_S>;
  using SB = std::integral_constant<int, TG_SUB>;
  using SR = std::integral_constant<int, TG_SBAR>;
  using SC = std::integral_constant<int, TG_SCALE>;
  AMG_CUDA_TRY(cudaMemsetAsync(w.sbar, 0, sizeof(double) * n, s));
  double total = 0.0;
  for (int j = 0; j < nsamples; ++j) {
    AMG_CUDA_TRY(cudaMemcpyAsync(w.e, e0 + (int64_t)j * n, sizeof(double) * n,
                                 cudaMemcpyDeviceToDevice, s));
    AMG_TRY(spmv(w.e, w.t));
    AMG_TRY(dot(w.e, w.t, 0));
    for (int k = 0; k < K; ++k) {
      AMG_TRY(smooth(w.e, w.a, w.Ae[k]));       // a = S e
      AMG_TRY(spmv(w.a, w.t));                   // c = a - P A_c^-1 P^T A a
      AMG_TRY(restrict_(w.t));
      AMG_TRY(csolve());
      AMG_TRY(vec(PS(), w.a, w.y, 0.0, w.c));
      AMG_TRY(smooth(w.c, w.e, w.Ac[k]));       // e = S c
    }
    AMG_TRY(spmv(w.e, w.t));
    AMG_TRY(dot(w.e, w.t, 1));
    AMG_CUDA_TRY(cudaMemcpyAsync(w.dots_host, w.dots, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                 s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    const double n0 = w.dots_host[0], nK = w.dots_host[1];
    if (!(n0 > 0.0) || !(nK > 0.0)) return AMG_ERR_NAN;
    total += 0.5 * log(nK / n0) / K;
    if (!domega) continue;
    // reverse pass; seed d/de_K = A e_K / (e_K^T A e_K) / (K nsamples)
    AMG_TRY(vec(SC(), w.t, nullptr, 1.0 / (nK * K * nsamples), w.eb));
    for (int k = K - 1; k >= 0; --k) {
      AMG_TRY(vec(SR(), w.eb, w.Ac[k], 0.0, w.sbar));   // sbar -= eb o (A c_k)
      AMG_TRY(vec(SS(), w.eb, nullptr, 0.0, w.t2));     // cb = S^T eb = eb - A (s o eb)
      AMG_TRY(spmv(w.t2, w.t));
      AMG_TRY(vec(SB(), w.eb, w.t, 0.0, w.cb));
      AMG_TRY(restrict_(w.cb));                          // ab = cb - A P A_c^-1 P^T cb
      AMG_TRY(csolve());
      AMG_TRY(vec(PR(), nullptr, w.y, 0.0, w.t2));
      AMG_TRY(spmv(w.t2, w.t));
      AMG_TRY(vec(SB(), w.cb, w.t, 0.0, w.ab));
      AMG_TRY(vec(SR(), w.ab, w.Ae[k], 0.0, w.sbar));   // sbar -= ab o (A e_k)
      AMG_TRY(vec(SS(), w.ab, nullptr, 0.0, w.t2));     // eb = S^T ab
      AMG_TRY(spmv(w.t2, w.t));
      AMG_TRY(vec(SB(), w.ab, w.t, 0.0, w.eb));
    }
  }
  *loss = total / nsamples;
  if (domega) {
    k_tg_vec<TG_DOMEGA><<<gv, 256, 0, s>>>(n, w.sbar, L0.d, nullptr, nullptr, 0.0, nullptr,
                                           domega);
    AMG_LAUNCH_CHECK();
  }
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  return AMG_OK;
}

}  // namespace amg
