// CSR -> sliced-ELL conversion and the plain FP64 SpMV (y = alpha A x + beta y).
#include "sellk.cuh"

namespace amg {

// Rows of slice s: [s*C, min(n, s*C + C)), or [row0[s], row0[s+1]) when the
// slices restart at every system boundary.
__device__ __forceinline__ void slice_rows(int64_t s, int C, int64_t n, const int64_t* row0,
                                           int64_t* b, int64_t* e) {
  if (row0) {
    *b = row0[s];
    *e = row0[s + 1];
  } else {
    *b = s * C;
    *e = (s + 1) * C < n ? (s + 1) * C : n;
  }
}

// Slice lengths (width * C) from the CSR row lengths.
__global__ void k_sell_widths(int64_t n, int64_t nslices, int C, const int64_t* row0,
                              const int64_t* rowptr, int64_t* slen) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  int64_t rb, re, w = 0;
  slice_rows(s, C, n, row0, &rb, &re);
  for (int64_t i = rb; i < re; ++i) {
    int64_t len = rowptr[i + 1] - rowptr[i];
    w = len > w ? len : w;
  }
  slen[s] = w * C;
}

// One thread per slot row of a slice: copy its entries, pad the rest.
__global__ void k_sell_fill(int64_t n, int64_t ncols, int64_t nslices, int C,
                            const int64_t* row0, const int64_t* rowptr, const int32_t* col,
                            const double* val, const int64_t* sliceptr, int32_t* ocol,
                            double* oval) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nslices * C) return;
  const int64_t s = t / C;
  const int r = (int)(t % C);
  int64_t sb, se;
  slice_rows(s, C, n, row0, &sb, &se);
  const int64_t i = sb + r;
  const int64_t beg = sliceptr[s];
  const int w = (int)((sliceptr[s + 1] - beg) / C);
  int64_t rb = 0, len = 0;
  if (i < se) {
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
                  const double* val, int C, int tpr, Sell& out, cudaStream_t s,
                  const std::vector<int64_t>* sys_off) {
  if (n <= 0 || ncols <= 0) return AMG_ERR_ARG;
  if (C * tpr != 32) return AMG_ERR_ARG;
  out.n = n;
  out.C = C;
  out.tpr = tpr;
  out.nslices = (n + C - 1) / C;
  if (sys_off && sys_off->size() >= 2) {  // batched systems: restart slices at each one
    std::vector<int64_t> row0;
    std::vector<int32_t> sys;
    for (size_t k = 0; k + 1 < sys_off->size(); ++k)
      for (int64_t r = (*sys_off)[k]; r < (*sys_off)[k + 1]; r += C) {
        row0.push_back(r);
        sys.push_back((int32_t)k);
      }
    if (sys_off->back() != n) return AMG_ERR_ARG;
    row0.push_back(n);
    out.nslices = (int64_t)sys.size();
    AMG_TRY(ar.alloc_n(&out.row0, out.nslices + 1));
    AMG_TRY(ar.alloc_n(&out.sys, out.nslices));
    AMG_CUDA_TRY(cudaMemcpyAsync(out.row0, row0.data(), sizeof(int64_t) * row0.size(),
                                 cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaMemcpyAsync(out.sys, sys.data(), sizeof(int32_t) * sys.size(),
                                 cudaMemcpyHostToDevice, s));
    AMG_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors go out of scope
  }
  int64_t* slen = nullptr;
  AMG_TRY(ar.alloc_n(&slen, out.nslices));
  AMG_TRY(ar.alloc_n(&out.sliceptr, out.nslices + 1));
  k_sell_widths<<<(unsigned)((out.nslices + 255) / 256), 256, 0, s>>>(n, out.nslices, C,
                                                                       out.row0, rowptr, slen);
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
  k_sell_fill<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(n, ncols, out.nslices, C, out.row0,
                                                             rowptr, col, val, out.sliceptr,
                                                             out.col, out.v64);
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
__global__ void __launch_bounds__(SELL_BLOCK, SELL_MIN_BLOCKS)
    k_spmv64(SellView<double> A, double alpha, const double* __restrict__ x, double beta,
             double* __restrict__ y) {
  const Lanes<TPR> ln;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < A.nslices;
       s += nw) {
    double acc = sell_row<TPR, double>(A, s, ln, [&](int j) { return __ldg(x + j); });
    const int64_t i = lane_row(A, s, ln);
    if (i >= 0) y[i] = beta == 0.0 ? alpha * acc : alpha * acc + beta * y[i];
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
