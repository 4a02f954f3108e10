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

// Slot layout of a slice.  Sorted: slot k of a row holds its k-th entry
// (ascending columns), padding after the last one.  Aligned: the slice's ELL
// columns are the distinct column offsets o = col - row of its rows, in
// ascending order, and a row places each entry in the column of its offset
// (padding where it has none), so a stencil's ELL column k holds one offset
// and its columns differ only by the row.  Aligned is used when the distinct
// offsets are no more than the longest row (no extra padding).  Either way a
// row's entries are visited in ascending column order with zero-valued
// padding in between, so every sum comes out the same.

// Distinct column offsets of rows [rb, re), ascending; writes them to `u`
// (if non-null) and returns their count, or -1 once it exceeds `cap`.
__device__ int slice_offsets(int64_t rb, int64_t re, const int64_t* rowptr, const int32_t* col,
                             int cap, int32_t* u) {
  int pos[64];  // rows of the slice: at most the largest slice height
  const int m = (int)(re - rb);
  for (int r = 0; r < m; ++r) pos[r] = 0;
  int cnt = 0;
  for (;;) {
    int64_t next = INT64_MAX;
    for (int r = 0; r < m; ++r) {
      const int64_t i = rb + r, len = rowptr[i + 1] - rowptr[i];
      if (pos[r] < len) {
        const int64_t o = (int64_t)col[rowptr[i] + pos[r]] - i;
        next = o < next ? o : next;
      }
    }
    if (next == INT64_MAX) return cnt;
    if (cnt == cap) return -1;
    if (u) u[cnt] = (int32_t)next;
    ++cnt;
    for (int r = 0; r < m; ++r) {
      const int64_t i = rb + r, len = rowptr[i + 1] - rowptr[i];
      if (pos[r] < len && (int64_t)col[rowptr[i] + pos[r]] - i == next) ++pos[r];
    }
  }
}

// Slice lengths (width * C) and the aligned flag of every slice.
__global__ void k_sell_widths(int64_t n, int64_t nslices, int C, const int64_t* row0,
                              const int64_t* rowptr, const int32_t* col, int64_t* slen,
                              uint8_t* aligned, int* wmax) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  int64_t rb, re, w = 0;
  slice_rows(s, C, n, row0, &rb, &re);
  for (int64_t i = rb; i < re; ++i) {
    int64_t len = rowptr[i + 1] - rowptr[i];
    w = len > w ? len : w;
  }
  aligned[s] = w > 0 && slice_offsets(rb, re, rowptr, col, (int)w, nullptr) >= 0;
  slen[s] = w * C;
  atomicMax(wmax, (int)(w < 0x7fffffff ? w : 0x7fffffff));
}

// Offsets of the aligned slices, stored per ELL column at sliceptr[s]/C + k.
__global__ void k_sell_offsets(int64_t n, int64_t nslices, int C, const int64_t* row0,
                               const int64_t* rowptr, const int32_t* col,
                               const int64_t* sliceptr, const uint8_t* aligned, int32_t* uoff) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices || !aligned[s]) return;
  int64_t rb, re;
  slice_rows(s, C, n, row0, &rb, &re);
  const int w = (int)((sliceptr[s + 1] - sliceptr[s]) / C);
  slice_offsets(rb, re, rowptr, col, w, uoff + sliceptr[s] / C);
}

// One thread per slot row of a slice: place its entries, pad the rest.
__global__ void k_sell_fill(int64_t n, int64_t ncols, int64_t nslices, int C,
                            const int64_t* row0, const int64_t* rowptr, const int32_t* col,
                            const double* val, const int64_t* sliceptr, const uint8_t* aligned,
                            const int32_t* uoff, int32_t* ocol, double* oval) {
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
  if (aligned[s]) {
    // ELL column k holds offset u[k]; padding reads column i + u[k] clamped
    // into range (value 0), which keeps the ELL column's columns together
    const int32_t* u = uoff + beg / C;
    const int64_t ir = i < se ? i : se - 1;
    int64_t e = 0;
    for (int k = 0; k < w; ++k) {
      const int64_t dst = beg + (int64_t)k * C + r;
      if (e < len && (int64_t)col[rb + e] - i == u[k]) {
        ocol[dst] = col[rb + e];
        oval[dst] = val[rb + e];
        ++e;
      } else {
        int64_t c = ir + u[k];
        c = c < 0 ? 0 : c >= ncols ? ncols - 1 : c;
        ocol[dst] = (int32_t)c;
        oval[dst] = 0.0;
      }
    }
    return;
  }
  // padding (value 0) reads a valid column: the row's last one (it is in
  // cache, and it keeps the slice's column deltas small), else the row itself
  const int32_t pad_col =
      len > 0 ? col[rb + len - 1] : (int32_t)(i < ncols ? i : ncols - 1);
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

// Column compression, one thread per slice: for each ELL column k the base is
// the smallest column of its C slots and every slot stores its offset from it.
// A slice whose offsets do not fit 16 bits raises *wide (the caller then
// keeps plain columns for the whole matrix).
__global__ void k_sell_compress(int64_t nslices, int C, const int64_t* sliceptr,
                                const int32_t* col, uint16_t* d16, int32_t* kbase, int* wide) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  const int64_t beg = sliceptr[s];
  const int w = (int)((sliceptr[s + 1] - beg) / C);
  for (int k = 0; k < w; ++k) {
    const int32_t* c = col + beg + (int64_t)k * C;
    int32_t lo = c[0], hi = c[0];
    for (int r = 1; r < C; ++r) {
      lo = c[r] < lo ? c[r] : lo;
      hi = c[r] > hi ? c[r] : hi;
    }
    if ((int64_t)hi - (int64_t)lo > 65535) *wide = 1;
    kbase[beg / C + k] = lo;
    for (int r = 0; r < C; ++r) d16[beg + (int64_t)k * C + r] = (uint16_t)(c[r] - lo);
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
                  const std::vector<int64_t>* sys_off, bool compress) {
  if (n <= 0 || ncols <= 0) return AMG_ERR_ARG;
  // heights 1..64 and 1..32 threads per row, powers of two; batched systems
  // keep one slice per warp (slice height x threads per row = 32)
  if (C < 1 || C > 64 || (C & (C - 1)) || tpr < 1 || tpr > 32 || (tpr & (tpr - 1)))
    return AMG_ERR_ARG;
  if (sys_off && sys_off->size() >= 2 && C * tpr != 32) return AMG_ERR_ARG;
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
  uint8_t* aligned = nullptr;
  int* wmax = nullptr;
  AMG_TRY(ar.alloc_n(&slen, out.nslices));
  AMG_TRY(ar.alloc_n(&aligned, out.nslices));
  AMG_TRY(ar.alloc_n(&wmax, 1));
  AMG_TRY(ar.alloc_n(&out.sliceptr, out.nslices + 1));
  AMG_CUDA_TRY(cudaMemsetAsync(wmax, 0, sizeof(int), s));
  const unsigned gs = (unsigned)((out.nslices + 127) / 128);
  k_sell_widths<<<gs, 128, 0, s>>>(n, out.nslices, C, out.row0, rowptr, col, slen, aligned,
                                   wmax);
  AMG_LAUNCH_CHECK();
  int wmax_h = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&wmax_h, wmax, sizeof(int), cudaMemcpyDeviceToHost, s));
  int64_t total = 0;
  AMG_TRY(scan_exclusive_i64(ar, slen, out.sliceptr, out.nslices, &total, s));
  AMG_CUDA_TRY(cudaMemcpyAsync(out.sliceptr + out.nslices, &total, sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
  ar.release(slen);
  ar.release(wmax);  // scan_exclusive_i64 synchronised: wmax_h is set
  out.wmax = wmax_h;
  out.nnz_pad = total;
  AMG_TRY(ar.alloc_n(&out.col, total));
  AMG_TRY(ar.alloc_n(&out.v64, total));
  int32_t* uoff = nullptr;
  AMG_TRY(ar.alloc_n(&uoff, total / C));
  k_sell_offsets<<<gs, 128, 0, s>>>(n, out.nslices, C, out.row0, rowptr, col, out.sliceptr,
                                    aligned, uoff);
  AMG_LAUNCH_CHECK();
  int64_t rows = out.nslices * C;
  k_sell_fill<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(n, ncols, out.nslices, C, out.row0,
                                                             rowptr, col, val, out.sliceptr,
                                                             aligned, uoff, out.col, out.v64);
  AMG_LAUNCH_CHECK();
  if (compress && tpr <= 8) AMG_TRY(sell_compress(ar, out, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  ar.release(aligned);
  ar.release(uoff);
  AMG_CUDA_TRY(cudaStreamSynchronize(s));  // `total` lives on this stack frame
  return AMG_OK;
}

int sell_compress(Arena& ar, Sell& A, cudaStream_t s) {
  int* wide = nullptr;
  AMG_TRY(ar.alloc_n(&A.d16, A.nnz_pad));
  AMG_TRY(ar.alloc_n(&A.kbase, A.nnz_pad / A.C));
  AMG_TRY(ar.alloc_n(&wide, 1));
  AMG_CUDA_TRY(cudaMemsetAsync(wide, 0, sizeof(int), s));
  k_sell_compress<<<(unsigned)((A.nslices + 127) / 128), 128, 0, s>>>(
      A.nslices, A.C, A.sliceptr, A.col, A.d16, A.kbase, wide);
  AMG_LAUNCH_CHECK();
  int h = 0;
  AMG_CUDA_TRY(cudaMemcpyAsync(&h, wide, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CUDA_TRY(cudaStreamSynchronize(s));
  ar.release(wide);
  if (h) {
    ar.release(A.d16);
    ar.release(A.kbase);
    A.d16 = nullptr;
    A.kbase = nullptr;
  }
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
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < A.ngroups;
       s += nw) {
    double acc = sell_row<TPR, double>(A, s, ln, [&](int j) { return __ldg(x + j); });
    const int64_t i = lane_row(A, s, ln);
    if (i >= 0) y[i] = beta == 0.0 ? alpha * acc : alpha * acc + beta * y[i];
  }
}

int sell_spmv64(const Sell& A, double alpha, const double* x, double beta, double* y,
                int num_sms, cudaStream_t s) {
  const int grid = sell_grid(sell_groups(A), num_sms);
  SellView<double> v = view(A, (const double*)A.v64);
  AMG_DISPATCH_TPR(sell_code(A),
                   (k_spmv64<TPR><<<grid, SELL_BLOCK, 0, s>>>(v, alpha, x, beta, y)));
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

}  // namespace amg
