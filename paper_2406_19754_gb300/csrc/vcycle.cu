// The V(1,1) cycle of Eq. (amg) with zero initial guess on every level:
//
//   x = S b;  r = b - A x;  b_c = P^T r;  x_c = V(b_c);  x += P x_c;
//   x += S (b - A x),       S = diag(s), s_i = omega_i / (l1 row sum)_i,
//
// where P is the 0/1 aggregate map, and the coarsest level is solved by its
// dense Cholesky factor.  Each level streams two operators built at setup,
//   Ah = A S   (a_ij s_j)  and  AP = A P  (row i, column J: sum of a_ij over
//   agg(j) = J),
// so that every matrix entry needs exactly one gathered vector element:
//   k_pre      r = b - Ah b                 (= b - A (S b): pre-smooth + residual)
//   k_restrict b_c[I] = sum of r_i over the members of I, ascending
//   k_post     z = S b + P x_c + S (r - AP x_c)
// The last line is y + S (b - A y) for y = S b + P x_c, because
// b - A y = (b - A S b) - A P x_c.  The level-0 k_post can also reduce (r, z)
// and (z, q) for the PCG step.
#include <algorithm>

#include "sellk.cuh"

namespace amg {

// ------------------------------------------------------------------ kernels

template <int TPR, typename V, typename T, typename BT>
__global__ void __launch_bounds__(SELL_BLOCK)
    k_pre(SellView<V> Ah, const BT* __restrict__ b, T* __restrict__ r) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < Ah.nslices;
       sl += nw) {
    const T acc =
        sell_row<TPR, T>(Ah, sl, ln, [&](int j) { return to_f(__ldg(b + j), T(0)); });
    const int64_t i = sl * Lanes<TPR>::C + ln.r;
    if (ln.t == 0 && i < Ah.n) r[i] = to_f(b[i], T(0)) - acc;
  }
}

template <typename T>
__global__ void k_restrict(int64_t nc, int stride, const int32_t* __restrict__ members,
                           const T* __restrict__ r, T* __restrict__ bc) {
  for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < nc;
       I += (int64_t)gridDim.x * blockDim.x) {
    const int32_t* m = members + I * stride;
    T acc = r[m[0]];
    for (int k = 1; k < stride; ++k) {
      const int32_t i = m[k];
      if (i < 0) break;
      acc = acc + r[i];
    }
    bc[I] = acc;
  }
}

// Epilogue of the level-0 post-smoother when it feeds PCG: t[0] = (r, z),
// t[1] = (z, q).  beta = (r+, z+)/(r, z) or, flexible, -(z+, q)/(p, q).
struct VcycleDotEpi {
  PcgScalars* sc;
  template <int NV>
  __device__ void operator()(double (&t)[NV]) const {
    const double rz = t[0];
    const double zq = NV > 1 ? t[NV > 1 ? 1 : 0] : 0.0;
    const double beta = sc->beta_form == PCG_BETA_FLEXIBLE ? -zq / sc->pq : rz / sc->rz;
    sc->beta = beta;
    sc->zq = zq;
    sc->rz = rz;
    if (!isfinite(rz) && sc->status == 0) sc->status = AMG_ERR_NAN;
  }
};

template <int TPR, typename V, typename T, typename BT, typename XT, int NDOT>
__global__ void __launch_bounds__(SELL_BLOCK)
    k_post(SellView<V> AP, const BT* __restrict__ b, const T* __restrict__ s,
           const T* __restrict__ r, const int32_t* __restrict__ agg, const T* __restrict__ xc,
           XT* __restrict__ x, const double* __restrict__ q, Reduce red, PcgScalars* sc) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double d[NDOT > 0 ? NDOT : 1];
#pragma unroll
  for (int k = 0; k < (NDOT > 0 ? NDOT : 1); ++k) d[k] = 0.0;
  for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < AP.nslices;
       sl += nw) {
    const T acc = sell_row<TPR, T>(AP, sl, ln, [&](int J) { return __ldg(xc + J); });
    const int64_t i = sl * Lanes<TPR>::C + ln.r;
    if (ln.t == 0 && i < AP.n) {
      const T bi = to_f(b[i], T(0));
      const T si = s[i];
      const T yi = si * bi + xc[agg[i]];
      const XT zi = to_f(yi + si * (r[i] - acc), XT(0));
      x[i] = zi;
      if (NDOT > 0) d[0] += (double)b[i] * (double)zi;
      if (NDOT > 1) d[NDOT > 1 ? 1 : 0] += (double)zi * q[i];
    }
  }
  if constexpr (NDOT > 0) grid_reduce<NDOT>(d, red, VcycleDotEpi{sc});
}

// Dots for the single-level case (the whole preconditioner is the coarse solve).
template <int NDOT>
__global__ void k_dots_rz(int64_t n, const double* r, const double* z, const double* q, Reduce red,
                          PcgScalars* sc) {
  double d[NDOT];
#pragma unroll
  for (int k = 0; k < NDOT; ++k) d[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    d[0] += r[i] * z[i];
    if (NDOT > 1) d[NDOT > 1 ? 1 : 0] += z[i] * q[i];
  }
  grid_reduce<NDOT>(d, red, VcycleDotEpi{sc});
}

// Coarsest level: x = L^-T (L^-1 b), one block, vectors staged in shared memory.
template <typename BT, typename XT>
__global__ void k_coarse(int n, const double* __restrict__ Linv, const double* __restrict__ LinvT,
                         const BT* __restrict__ b, XT* __restrict__ x) {
  extern __shared__ double csh[];
  double* bs = csh;
  double* ys = csh + n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) bs[i] = (double)b[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = w; i < n; i += nw) {
    double acc = 0.0;
    const double* row = Linv + (int64_t)i * n;
    for (int k = lane; k <= i; k += 32) acc += row[k] * bs[k];
    acc = warp_sum(acc);
    if (lane == 0) ys[i] = acc;
  }
  __syncthreads();
  for (int k = w; k < n; k += nw) {
    double acc = 0.0;
    const double* row = LinvT + (int64_t)k * n;
    for (int i = k + lane; i < n; i += 32) acc += row[i] * ys[i];
    acc = warp_sum(acc);
    if (lane == 0) x[k] = (XT)acc;
  }
}

// ------------------------------------------------------------------ driver

template <typename BT, typename XT>
static int coarse_solve(const amg_handle* H, const BT* b, XT* x, cudaStream_t s) {
  const int n = (int)H->nco;
  const size_t sm = sizeof(double) * 2 * (size_t)n;  // n <= 3072 keeps this under 48 KB
  k_coarse<BT, XT><<<1, 1024, sm, s>>>(n, H->Linv, H->LinvT, b, x);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

template <typename V, typename T, typename BT>
static int launch_pre(const amg_handle* H, const Level& L, const V* ah, const BT* b, T* r,
                      cudaStream_t s) {
  const int grid = sell_grid(L.A.nslices, H->num_sms);
  const SellView<V> v = view<V>(L.A, ah);
  AMG_DISPATCH_TPR(L.A.tpr, (k_pre<TPR, V, T, BT><<<grid, SELL_BLOCK, 0, s>>>(v, b, r)));
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

template <typename V, typename T, typename BT, typename XT, int NDOT>
static int launch_post(const amg_handle* H, const Level& L, const V* ap, const BT* b,
                       const T* xc, XT* x, const double* q, cudaStream_t s) {
  const int grid = sell_grid(L.AP.nslices, H->num_sms);
  const SellView<V> v = view<V>(L.AP, ap);
  const T* sc = (const T*)(sizeof(T) == 8 ? (const void*)L.s64 : (const void*)L.s32);
  AMG_DISPATCH_TPR(L.AP.tpr, (k_post<TPR, V, T, BT, XT, NDOT><<<grid, SELL_BLOCK, 0, s>>>(
                                 v, b, sc, (const T*)L.r, L.agg, xc, x, q, H->red, H->sc)));
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

template <typename T>
static int launch_restrict(const amg_handle* H, const Level& L, const T* r, T* bc,
                           cudaStream_t s) {
  k_restrict<T><<<grid_for(L.nc, 256, H->num_sms, 8), 256, 0, s>>>(L.nc, L.stride, L.members, r,
                                                                   bc);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

template <typename BT>
static int pre_f32(const amg_handle* H, const Level& L, const BT* b, float* r, cudaStream_t s) {
  if (L.vstore == VAL_BF16) return launch_pre<__nv_bfloat16, float, BT>(H, L, L.ah16, b, r, s);
  return launch_pre<float, float, BT>(H, L, L.ah32, b, r, s);
}

template <typename T, typename BT, typename XT, int NDOT>
static int post_any(const amg_handle* H, const Level& L, const BT* b, const T* xc, XT* x,
                    const double* q, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    return launch_post<double, T, BT, XT, NDOT>(H, L, L.AP.v64, b, xc, x, q, s);
  } else {
    if (L.vstore == VAL_BF16)
      return launch_post<__nv_bfloat16, T, BT, XT, NDOT>(H, L, L.AP.v16, b, xc, x, q, s);
    return launch_post<float, T, BT, XT, NDOT>(H, L, L.AP.v32, b, xc, x, q, s);
  }
}

// Optional per-kernel timing: an event pair around every launch plus the
// kernel's algorithmic bytes (each array counted once per pass).
struct Prof {
  cudaStream_t s;
  std::vector<cudaEvent_t> ev;
  std::vector<amg_kernel_time> rec;
  int begin(int level, int kind, double bytes) {
    cudaEvent_t a, b;
    AMG_CUDA_TRY(cudaEventCreate(&a));
    AMG_CUDA_TRY(cudaEventCreate(&b));
    ev.push_back(a);
    ev.push_back(b);
    amg_kernel_time k;
    k.level = level;
    k.kind = kind;
    k.bytes = bytes;
    k.ms = 0.0;
    rec.push_back(k);
    AMG_CUDA_TRY(cudaEventRecord(a, s));
    return AMG_OK;
  }
  int end() {
    AMG_CUDA_TRY(cudaEventRecord(ev.back(), s));
    return AMG_OK;
  }
  int finish() {
    AMG_CUDA_TRY(cudaStreamSynchronize(s));
    for (size_t k = 0; k < rec.size(); ++k) {
      float ms = 0.f;
      AMG_CUDA_TRY(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
      rec[k].ms = ms;
    }
    return AMG_OK;
  }
  ~Prof() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

// Algorithmic bytes of each V-cycle kernel on one level: operator entries
// (value + int32 column) once, every vector once.  mb = bytes of an operator
// entry, vb = bytes of a V-cycle vector element, ib/ob = bytes of the level's
// input b / output z elements (FP64 on level 0).
static double bytes_pre(const Level& L, double mb, double vb, double ib) {
  return (double)L.nnz * mb + (double)L.n * (ib + vb);  // Ah, b, r
}
static double bytes_restrict(const Level& L, double vb) {
  return (double)L.n * (vb + 4.0) + (double)L.nc * vb;  // r, members, b_c
}
static double bytes_post(const Level& L, double mb, double vb, double ib, double ob) {
  // AP, b, s, r, agg, z, x_c
  return (double)L.ap_nnz * mb + (double)L.n * (ib + vb + vb + 4.0 + ob) + (double)L.nc * vb;
}

#define PROF_BEGIN(lvl, kind, bytes) \
  if (prof) AMG_TRY(prof->begin((lvl), (kind), (bytes)))
#define PROF_END() \
  if (prof) AMG_TRY(prof->end())

template <typename T>
static int vcycle_levels(const amg_handle* H, const double* r0, double* z0, int dots,
                         const double* q, cudaStream_t s, Prof* prof) {
  const int nl = (int)H->L.size();
  const double vb = sizeof(T);
  auto mbytes = [&](const Level& L) {
    return 4.0 + (L.vstore == VAL_F64 ? 8.0 : L.vstore == VAL_F32 ? 4.0 : 2.0);
  };
  if (nl == 1) {
    const double m = (double)H->nco;
    PROF_BEGIN(0, 3, m * m * 8.0 + m * 16.0);
    AMG_TRY(coarse_solve<double, double>(H, r0, z0, s));
    PROF_END();
    if (dots > 0) {
      const int grid = grid_for(H->L[0].n, 256, H->num_sms, 8);
      if (dots == 1)
        k_dots_rz<1><<<grid, 256, 0, s>>>(H->L[0].n, r0, z0, q, H->red, H->sc);
      else
        k_dots_rz<2><<<grid, 256, 0, s>>>(H->L[0].n, r0, z0, q, H->red, H->sc);
      AMG_LAUNCH_CHECK();
    }
    return AMG_OK;
  }
  // downward: pre-smooth + residual, restriction
  for (int l = 0; l < nl - 1; ++l) {
    const Level& L = H->L[l];
    T* r = (T*)L.r;
    PROF_BEGIN(l, 0, bytes_pre(L, mbytes(L), vb, l == 0 ? 8.0 : vb));
    if constexpr (sizeof(T) == 8) {
      const double* b = l == 0 ? r0 : (const double*)L.b;
      AMG_TRY((launch_pre<double, double, double>(H, L, L.ah64, b, r, s)));
    } else {
      if (l == 0)
        AMG_TRY(pre_f32<double>(H, L, r0, r, s));
      else
        AMG_TRY(pre_f32<float>(H, L, (const float*)L.b, r, s));
    }
    PROF_END();
    PROF_BEGIN(l, 1, bytes_restrict(L, vb));
    AMG_TRY(launch_restrict<T>(H, L, r, (T*)H->L[l + 1].b, s));
    PROF_END();
  }
  {
    const double m = (double)H->nco;
    PROF_BEGIN(nl - 1, 3, m * m * 8.0 + m * 2.0 * vb);
    AMG_TRY((coarse_solve<T, T>(H, (const T*)H->L[nl - 1].b, (T*)H->L[nl - 1].x, s)));
    PROF_END();
  }
  // upward: prolongation + post-smooth
  for (int l = nl - 2; l >= 1; --l) {
    const Level& L = H->L[l];
    PROF_BEGIN(l, 2, bytes_post(L, mbytes(L), vb, vb, vb));
    AMG_TRY((post_any<T, T, T, 0>(H, L, (const T*)L.b, (const T*)H->L[l + 1].x, (T*)L.x, q, s)));
    PROF_END();
  }
  const Level& L0 = H->L[0];
  const T* xc = (const T*)H->L[1].x;
  PROF_BEGIN(0, 2, bytes_post(L0, mbytes(L0), vb, 8.0, 8.0));
  int rc;
  if (dots == 0)
    rc = post_any<T, double, double, 0>(H, L0, r0, xc, z0, q, s);
  else if (dots == 1)
    rc = post_any<T, double, double, 1>(H, L0, r0, xc, z0, q, s);
  else
    rc = post_any<T, double, double, 2>(H, L0, r0, xc, z0, q, s);
  AMG_TRY(rc);
  PROF_END();
  return AMG_OK;
}

int vcycle_run(const amg_handle* H, const double* r, double* z, int dots, const double* q,
               cudaStream_t s) {
  if (H->opt.precision == AMG_PREC_F32) return vcycle_levels<float>(H, r, z, dots, q, s, nullptr);
  return vcycle_levels<double>(H, r, z, dots, q, s, nullptr);
}

int vcycle_profile(const amg_handle* H, const double* r, double* z, amg_kernel_time* out,
                   int max_out, int* count, cudaStream_t s) {
  Prof prof;
  prof.s = s;
  int rc = H->opt.precision == AMG_PREC_F32
               ? vcycle_levels<float>(H, r, z, 0, nullptr, s, &prof)
               : vcycle_levels<double>(H, r, z, 0, nullptr, s, &prof);
  AMG_TRY(rc);
  AMG_TRY(prof.finish());
  const int m = (int)prof.rec.size();
  if (count) *count = m;
  for (int k = 0; k < m && k < max_out; ++k) out[k] = prof.rec[k];
  return AMG_OK;
}

}  // namespace amg
