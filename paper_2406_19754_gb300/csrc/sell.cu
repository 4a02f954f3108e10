// CSR -> sliced-ELL conversion and the plain FP64 SpMV (y = alpha A x + beta y).
#include "sellk.cuh"

namespace amg {

// Slice lengths (width * C) from the CSR row lengths.
__global__ void k_sell_widths(int64_t n, int64_t nslices, int C, const int64_t* rowptr,
                              int64_t* slen) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  int64_t w = 0;
  for (int r = 0; r < C; ++r) {
    int64_t i = s * C + r;
    if (i < n) {
      int64_t len = rowptr[i + 1] - rowptr[i];
      w = len > w ? len : w;
    }
  }
  slen[s] = w * C;
}

// One thread per (padded) row: copy its entries into the slice, pad the rest.
__global__ void k_sell_fill(int64_t n, int64_t ncols, int64_t nslices, int C,
                            const int64_t* rowptr, const int32_t* col, const double* val,
                            const int64_t* sliceptr, int32_t* ocol, double* oval) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nslices * C) return;
  const int64_t s = i / C;
  const int r = (int)(i % C);
  const int64_t beg = sliceptr[s];
  const int w = (int)((sliceptr[s + 1] - beg) / C);
  int64_t rb = 0, len = 0;
  if (i < n) {
    rb = rowptr[i];
    len = rowptr[i + 1] - rowptr[i];
  }
  // padding reads a valid column: the row itself when it exists in x
  const int32_t pad_col = (int32_t)(i < ncols ? i : ncols - 1);
  for (int k = 0; k < w; ++k) {
    int64_t dst = beg + (int64_t)k * C + r;
    if (k < len) {
      ocol[dst] = col[rb + k];
      oval[dst] = val[rb + k];
    } else {
      ocol[dst] = pad_col;
      oval[dst] = 0.0;
    }
  }
}

__global__ void k_to_f32(int64_t n, const double* in, float* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

__global__ void k_to_bf16(int64_t n, const double* in, __nv_bfloat16* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn((float)in[i]);
}

int sell_from_csr(Arena& ar, int64_t n, int64_t ncols, const int64_t* rowptr, const int32_t* col,
                  const double* val, int C, int tpr, Sell& out, cudaStream_t s) {
  if (n <= 0 || ncols <= 0) return AMG_ERR_ARG;
  if (C * tpr != 32) return AMG_ERR_ARG;
  out.n = n;
  out.C = C;
  out.tpr = tpr;
  out.nslices = (n + C - 1) / C;
  int64_t* slen = nullptr;
  AMG_TRY(ar.alloc_n(&slen, out.nslices));
  AMG_TRY(ar.alloc_n(&out.sliceptr, out.nslices + 1));
  k_sell_widths<<<(unsigned)((out.nslices + 255) / 256), 256, 0, s>>>(n, out.nslices, C, rowptr,
                                                                       slen);
  AMG_LAUNCH_CHECK();
  int64_t total = 0;
  AMG_TRY(scan_exclusive_i64(ar, slen, out.sliceptr, out.nslices, &total, s));
  AMG_CUDA_TRY(cudaMemcpyAsync(out.sliceptr + out.nslices, &total, sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
  ar.release(slen);
  out.nnz_pad = total;
  AMG_TRY(ar.alloc_n(&out.col, total));
  AMG_TRY(ar.alloc_n(&out.v64, total));
  int64_t rows = out.nslices * C;
  k_sell_fill<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(n, ncols, out.nslices, C, rowptr,
                                                             col, val, out.sliceptr, out.col,
                                                             out.v64);
  AMG_LAUNCH_CHECK();
  AMG_CUDA_TRY(cudaStreamSynchronize(s));  // `total` lives on this stack frame
  return AMG_OK;
}

int sell_make_copies(Arena& ar, Sell& A, int vstore, cudaStream_t s) {
  if (vstore == VAL_F32 && !A.v32) {
    AMG_TRY(ar.alloc_n(&A.v32, A.nnz_pad));
    k_to_f32<<<1024, 256, 0, s>>>(A.nnz_pad, A.v64, A.v32);
    AMG_LAUNCH_CHECK();
  }
  if (vstore == VAL_BF16 && !A.v16) {
    AMG_TRY(ar.alloc_n(&A.v16, A.nnz_pad));
    k_to_bf16<<<1024, 256, 0, s>>>(A.nnz_pad, A.v64, A.v16);
    AMG_LAUNCH_CHECK();
  }
  return AMG_OK;
}

template <int TPR>
__global__ void __launch_bounds__(SELL_BLOCK)
    k_spmv64(SellView<double> A, double alpha, const double* __restrict__ x, double beta,
             double* __restrict__ y) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < A.nslices;
       s += nw) {
    double acc = sell_row<TPR, double>(A, s, ln, [&](int j) { return __ldg(x + j); });
    const int64_t i = s * Lanes<TPR>::C + ln.r;
    if (ln.t == 0 && i < A.n) y[i] = beta == 0.0 ? alpha * acc : alpha * acc + beta * y[i];
  }
}

int sell_spmv64(const Sell& A, double alpha, const double* x, double beta, double* y,
                int num_sms, cudaStream_t s) {
  const int grid = sell_grid(A.nslices, num_sms);
  SellView<double> v = view(A, (const double*)A.v64);
  AMG_DISPATCH_TPR(A.tpr, (k_spmv64<TPR><<<grid, SELL_BLOCK, 0, s>>>(v, alpha, x, beta, y)));
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

}  // namespace amg
