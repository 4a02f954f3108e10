// Learned smoother weights: a 9 -> 32 -> 32 -> 1 MLP (GELU hidden layers,
// output omega = max(omega_max sigmoid(z), 1e-3) with omega_max 1 by default
// or in (1, 2) by mlp_set_omega_max) maps per-row stencil features to the l1-Jacobi
// damping weight omega_i (s_i = omega_i / d_i, Sec. 2.3 l1-Jacobi; the network
// is not in the paper).  FP32 weights and activations; gradients are summed
// in FP64 with a fixed order (per-block partials, then blocks in order), so
// training is reproducible run to run.
//
// Parameter layout (1409 floats): W1[32][9], b1[32], W2[32][32], b2[32],
// W3[32], b3.
#include <math.h>

#include <algorithm>
#include <vector>

#include <cuda_fp16.h>

#include "common.cuh"

namespace amg {

constexpr int NF = 9, NH = 32;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NF, OFF_W2 = OFF_B1 + NH,
              OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH,
              NPARAM = OFF_B3 + 1;
constexpr float OMEGA_MIN = 1e-3f;
constexpr int BW_ROWS = 64;  // rows staged per backward chunk (one thread each)
constexpr int BW_BLOCKS_MAX = 1024;

}  // namespace amg

struct mlp_handle {
  float omega_max = 1.0f;  // output cap: omega = max(omega_max * sigmoid(z), OMEGA_MIN)
  int exact = 0;           // 1: the FP32 CUDA-core forward pass instead of the tensor cores
  float* params = nullptr;
  double* grad = nullptr;   // accumulated gradient (FP64)
  double* gpart = nullptr;  // per-block partial gradients
  double* m = nullptr;      // Adam moments
  double* v = nullptr;
  int t = 0;
  int num_sms = 0;
  int tc_blocks = 0;  // resident CTAs of the tensor-core forward pass on this GPU
  amg::Arena arena;
};

namespace amg {

__device__ __forceinline__ float gelu_f(float u) {
  return 0.5f * u * (1.0f + erff(u * 0.70710678f));
}
__device__ __forceinline__ float gelu_df(float u) {
  return 0.5f * (1.0f + erff(u * 0.70710678f)) + u * expf(-0.5f * u * u) * 0.39894228f;
}

// Features of row i of a 7-point operator on an nx x ny x nz grid:
// a_ij / a_ii towards -x, +x, -y, +y, -z, +z (0 if absent), the l1 ratio,
// log(max|a_ij| / min|a_ij|) and the neighbour count / 6.  FP32 arithmetic
// on the FP64 entries (the features are FP32; GB300's FP64 pipe made the
// divisions and the logarithm the cost of this kernel): one reciprocal of
// a_ii, and the logarithm as log1p((max - min) / min), which stays accurate
// when max and min are close.
__device__ __forceinline__ void row_features(int64_t i, int64_t nx, int64_t nxy,
                                             const int64_t* __restrict__ rp,
                                             const int32_t* __restrict__ ci,
                                             const double* __restrict__ v, float (&f)[NF]) {
  const int64_t e0 = rp[i], e1 = rp[i + 1];
  float aii = 0.0f;
  for (int64_t e = e0; e < e1; ++e)
    if (ci[e] == i) aii = (float)v[e];
  const float inv = 1.0f / aii;
  float off[6] = {0, 0, 0, 0, 0, 0}, l1 = 0.0f, amax = 0.0f, amin = 0.0f;
  int cnt = 0;
  for (int64_t e = e0; e < e1; ++e) {
    const int64_t d = (int64_t)ci[e] - i;
    if (d == 0) continue;
    const float a = (float)v[e];
    int slot = -1;
    if (d == -1) slot = 0;
    else if (d == 1) slot = 1;
    else if (d == -nx) slot = 2;
    else if (d == nx) slot = 3;
    else if (d == -nxy) slot = 4;
    else if (d == nxy) slot = 5;
    if (slot >= 0) off[slot] = a * inv;
    const float m = fabsf(a);
    l1 += m;
    amax = cnt == 0 ? m : fmaxf(amax, m);
    amin = cnt == 0 ? m : fminf(amin, m);
    ++cnt;
  }
  for (int k = 0; k < 6; ++k) f[k] = off[k];
  f[6] = l1 * inv;
  f[7] = (cnt > 0 && amin > 0.0f) ? log1pf((amax - amin) / amin) : 0.0f;
  f[8] = (float)cnt / 6.0f;
}

__global__ void k_features(int64_t n, int64_t nx, int64_t nxy, const int64_t* __restrict__ rp,
                           const int32_t* __restrict__ ci, const double* __restrict__ v,
                           float* __restrict__ feat) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float f[NF];
    row_features(i, nx, nxy, rp, ci, v, f);
    for (int k = 0; k < NF; ++k) feat[i * NF + k] = f[k];
  }
}

struct RowAct {
  float u1[NH], h1[NH], u2[NH], h2[NH], z, sg;
};

__device__ __forceinline__ void mlp_row(const float* __restrict__ p, const float* f, RowAct& a) {
#pragma unroll 4
  for (int o = 0; o < NH; ++o) {
    float s = p[OFF_B1 + o];
#pragma unroll
    for (int i = 0; i < NF; ++i) s = fmaf(p[OFF_W1 + o * NF + i], f[i], s);
    a.u1[o] = s;
    a.h1[o] = gelu_f(s);
  }
  for (int o = 0; o < NH; ++o) {
    float s = p[OFF_B2 + o];
#pragma unroll 8
    for (int i = 0; i < NH; ++i) s = fmaf(p[OFF_W2 + o * NH + i], a.h1[i], s);
    a.u2[o] = s;
    a.h2[o] = gelu_f(s);
  }
  float z = p[OFF_B3];
#pragma unroll 8
  for (int i = 0; i < NH; ++i) z = fmaf(p[OFF_W3 + i], a.h2[i], z);
  a.z = z;
  a.sg = 1.0f / (1.0f + expf(-z));
}

// Forward pass by tiles of 32 rows, one warp per tile: lane o evaluates
// neuron o of each layer for the tile's rows with its weights in registers;
// the tile's features and activations sit in shared memory and are read as
// broadcasts (four at a time where rows are 16-byte aligned), so no weight is
// re-read per row.  Each output is the same chain of fmaf calls, in the same
// order, as mlp_row, so omega is the same bits as a thread-per-row pass.
constexpr int FW_WARPS = 4;
constexpr int FW_FLD = 12;  // padded feature row (3 float4)
constexpr int FW_HLD = 36;  // padded activation row (float4-aligned, fewer conflicts)

__global__ void __launch_bounds__(FW_WARPS * 32)
    k_mlp_forward_tiled(int64_t n, const float* __restrict__ params,
                        const float* __restrict__ feat, float omega_max,
                        float* __restrict__ omega) {
  __shared__ __align__(16) float fs[FW_WARPS][32 * FW_FLD];
  __shared__ __align__(16) float hs[FW_WARPS][32 * FW_HLD];
  __shared__ float zs[FW_WARPS][32 * 33];
  __shared__ float w3s[NH];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float w1[NF], w2[NH];
#pragma unroll
  for (int i = 0; i < NF; ++i) w1[i] = params[OFF_W1 + lane * NF + i];
#pragma unroll
  for (int i = 0; i < NH; ++i) w2[i] = params[OFF_W2 + lane * NH + i];
  const float b1 = params[OFF_B1 + lane], b2 = params[OFF_B2 + lane], b3 = params[OFF_B3];
  if (threadIdx.x < NH) w3s[threadIdx.x] = params[OFF_W3 + threadIdx.x];
  __syncthreads();
  float* f = fs[w];
  float* h = hs[w];
  float* zr = zs[w];
  const int64_t ntiles = (n + 31) / 32;
  for (int64_t t = (int64_t)blockIdx.x * FW_WARPS + w; t < ntiles;
       t += (int64_t)gridDim.x * FW_WARPS) {
    const int64_t r0 = t * 32;
    const int rows = (int)(n - r0 < 32 ? n - r0 : 32);
    for (int k = lane; k < rows * NF; k += 32) f[(k / NF) * FW_FLD + k % NF] = feat[r0 * NF + k];
    __syncwarp();
    for (int r = 0; r < rows; ++r) {  // layer 1
      const float4 fa = *(const float4*)(f + r * FW_FLD);
      const float4 fb = *(const float4*)(f + r * FW_FLD + 4);
      const float f8 = f[r * FW_FLD + 8];
      float s = b1;
      s = fmaf(w1[0], fa.x, s);
      s = fmaf(w1[1], fa.y, s);
      s = fmaf(w1[2], fa.z, s);
      s = fmaf(w1[3], fa.w, s);
      s = fmaf(w1[4], fb.x, s);
      s = fmaf(w1[5], fb.y, s);
      s = fmaf(w1[6], fb.z, s);
      s = fmaf(w1[7], fb.w, s);
      s = fmaf(w1[8], f8, s);
      h[r * FW_HLD + lane] = gelu_f(s);
    }
    __syncwarp();
    for (int r = 0; r < rows; ++r) {  // layer 2, and the products of layer 3
      float s = b2;
#pragma unroll
      for (int i = 0; i < NH; i += 4) {
        const float4 hv = *(const float4*)(h + r * FW_HLD + i);
        s = fmaf(w2[i], hv.x, s);
        s = fmaf(w2[i + 1], hv.y, s);
        s = fmaf(w2[i + 2], hv.z, s);
        s = fmaf(w2[i + 3], hv.w, s);
      }
      zr[r * 33 + lane] = gelu_f(s);
    }
    __syncwarp();
    if (lane < rows) {  // layer 3: lane r finishes row r
      float z = b3;
#pragma unroll 8
      for (int i = 0; i < NH; ++i) z = fmaf(w3s[i], zr[lane * 33 + i], z);
      const float sg = 1.0f / (1.0f + expf(-z));
      omega[r0 + lane] = fmaxf(omega_max * sg, OMEGA_MIN);
    }
    __syncwarp();
  }
}

// Forward pass on the tensor cores: the 9 -> 32 and 32 -> 32 layers of a tile
// of 16 rows are warp-level matrix products (mma.sync m16n8k16 with FP16
// operands rounded to nearest, FP32 accumulation); GELU, the 32 -> 1 layer
// and the sigmoid run in FP32 on the accumulators.  FP16 keeps 10 explicit
// mantissa bits, as TF32 does, at half the register cost per operand.
// Fragment layouts of m16n8k16 (g = lane / 4, t = lane % 4; a register holds
// two FP16 values, the lower column in its low half):
//   A (16 x 16, row major): a0 = (g, 2t..2t+1), a1 = (g+8, 2t..2t+1),
//                           a2 = (g, 2t+8..2t+9), a3 = (g+8, 2t+8..2t+9);
//   B (16 x 8, k x n):      b0 = (2t..2t+1, g), b1 = (2t+8..2t+9, g);
//   C (16 x 8, FP32):       c0 = (g, 2t), c1 = (g, 2t+1), c2 = (g+8, 2t),
//                           c3 = (g+8, 2t+1).
// The C fragments of the first layer's column tiles 2s and 2s+1 hold, for
// rows g and g+8, exactly the hidden units 16s + {2t, 2t+1, 2t+8, 2t+9} that
// the A fragment of the second layer's k-step s needs, so the activations
// pass from one product to the next in registers.  The features come
// straight from global memory into the first A fragment (columns 9..15 are
// zero); the weights stay in registers as B fragments for the whole launch.
// GELU uses gelu_fast.  omega agrees with the FP32 pass to about 1e-3.
constexpr int TC_WARPS = 4;

// GELU with erf by Abramowitz & Stegun, Handbook of Mathematical Functions,
// formula 7.1.26: for x >= 0, erf(x) = 1 - P(t) e^(-x^2), P(t) = a1 t + a2
// t^2 + a3 t^3 + a4 t^4 + a5 t^5, t = 1 / (1 + p x), |error| <= 1.5e-7; odd in
// x.  With x = u / sqrt(2), sign(x) u = |u| turns 0.5 u (1 + erf(x)) into
//   GELU(u) = max(u, 0) - |u| (P(t) / 2) e^(-u^2 / 2),  t = 1 / (1 + p |u| / sqrt(2)),
// which needs no sign transfer: a hardware reciprocal and base-2 exponential
// (rcp.approx, ex2.approx; e^y = 2^(y log2 e)), six FMAs and four other
// operations.  The tensor-core forward pass, whose FP16 operands already
// limit omega to about 1e-3, uses it in its GELUs.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float gelu_fast(float u) {
  const float ax = fabsf(u);
  const float t = rcp_approx(fmaf(0.3275911f * 0.70710678f, ax, 1.0f));
  // P(t) / 2, the coefficients a1..a5 halved
  const float q = t * fmaf(fmaf(fmaf(fmaf(0.5307027145f, t, -0.7265760135f), t, 0.7107068705f),
                                t, -0.142248368f),
                           t, 0.127414796f);
  const float e = ex2_approx(u * (u * (-0.5f * 1.44269504f)));
  return fmaf(-(ax * q), e, fmaxf(u, 0.0f));
}

// two floats rounded to FP16 (nearest even), lo in the low half
__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// d = A B + c (c is read, d written: a bias can enter as c without a copy)
__device__ __forceinline__ void mma_f16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                        uint32_t a3, uint32_t b0, uint32_t b1, float c0, float c1,
                                        float c2, float c3) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%10,%11,%12,%13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(c0), "f"(c1), "f"(c2),
        "f"(c3));
}

// The next tile's features are loaded into registers while the current one
// is computed.
__global__ void __launch_bounds__(TC_WARPS * 32, 5)
    k_mlp_forward_tc(int64_t n, const float* __restrict__ params,
                     const float* __restrict__ feat, float omega_max,
                     float* __restrict__ omega) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  // B fragments: W1^T (k = feature, n = neuron; k >= 9 is zero) and W2^T
  uint32_t w1b[4][2], w2b[2][4][2];
  float b1v[4][2], b2v[4][2], w3v[4][2];
  auto w1 = [&](int o, int k) { return k < NF ? params[OFF_W1 + o * NF + k] : 0.0f; };
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int o = 8 * nt + g;
    w1b[nt][0] = pack_h2(w1(o, 2 * t), w1(o, 2 * t + 1));
    w1b[nt][1] = pack_h2(w1(o, 2 * t + 8), w1(o, 2 * t + 9));
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const float* wr = params + OFF_W2 + o * NH + 16 * ks + 2 * t;
      w2b[ks][nt][0] = pack_h2(wr[0], wr[1]);
      w2b[ks][nt][1] = pack_h2(wr[8], wr[9]);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {  // this thread's accumulator columns 8 nt + 2 t + j
      b1v[nt][j] = params[OFF_B1 + 8 * nt + 2 * t + j];
      b2v[nt][j] = params[OFF_B2 + 8 * nt + 2 * t + j];
      w3v[nt][j] = params[OFF_W3 + 8 * nt + 2 * t + j];
    }
  }
  const float b3 = params[OFF_B3];
  const int64_t ntiles = (n + 15) / 16;
  const int64_t step = (int64_t)gridDim.x * TC_WARPS;
  // this lane's features of a tile: rows g and g + 8, columns 2t, 2t + 1 and
  // (lanes with t == 0) column 8; 0 beyond the last row
  auto load_tile = [&](int64_t tl, float (&v)[6]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t row = tl * 16 + g + 8 * h;
      const bool ok = tl < ntiles && row < n;
      const float* fr = feat + row * NF;
      v[3 * h] = ok ? __ldg(fr + 2 * t) : 0.0f;
      v[3 * h + 1] = ok ? __ldg(fr + 2 * t + 1) : 0.0f;
      v[3 * h + 2] = (ok && t == 0) ? __ldg(fr + 8) : 0.0f;
    }
  };
  float nxt[6];
  load_tile((int64_t)blockIdx.x * TC_WARPS + w, nxt);
  for (int64_t tile = (int64_t)blockIdx.x * TC_WARPS + w; tile < ntiles; tile += step) {
    const int64_t r0 = tile * 16;
    const int rows = (int)(n - r0 < 16 ? n - r0 : 16);
    const uint32_t f0 = pack_h2(nxt[0], nxt[1]), f1 = pack_h2(nxt[3], nxt[4]),
                   f2 = pack_h2(nxt[2], 0.0f), f3 = pack_h2(nxt[5], 0.0f);
    load_tile(tile + step, nxt);
    // layer 1: U1 = F W1^T + b1 (4 column tiles of 8, K = 16 with zeros beyond 9)
    float c1[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
      mma_f16(c1[nt], f0, f1, f2, f3, w1b[nt][0], w1b[nt][1], b1v[nt][0], b1v[nt][1],
              b1v[nt][0], b1v[nt][1]);
    // layer 2: U2 = GELU(U1) W2^T + b2, the A fragments straight from c1
    float c2[4][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const float(&lo)[4] = c1[2 * ks];
      const float(&hi)[4] = c1[2 * ks + 1];
      const uint32_t a0 = pack_h2(gelu_fast(lo[0]), gelu_fast(lo[1]));
      const uint32_t a1 = pack_h2(gelu_fast(lo[2]), gelu_fast(lo[3]));
      const uint32_t a2 = pack_h2(gelu_fast(hi[0]), gelu_fast(hi[1]));
      const uint32_t a3 = pack_h2(gelu_fast(hi[2]), gelu_fast(hi[3]));
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        if (ks == 0)
          mma_f16(c2[nt], a0, a1, a2, a3, w2b[0][nt][0], w2b[0][nt][1], b2v[nt][0], b2v[nt][1],
                  b2v[nt][0], b2v[nt][1]);
        else
          mma_f16(c2[nt], a0, a1, a2, a3, w2b[1][nt][0], w2b[1][nt][1], c2[nt][0], c2[nt][1],
                  c2[nt][2], c2[nt][3]);
      }
    }
    // z = GELU(U2) w3 + b3 per row
    float zg = 0.0f, zg8 = 0.0f;  // partial z of rows g and g + 8 over this thread's columns
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        zg = fmaf(w3v[nt][j], gelu_fast(c2[nt][j]), zg);
        zg8 = fmaf(w3v[nt][j], gelu_fast(c2[nt][2 + j]), zg8);
      }
    // the four threads of a group hold a row's 32 columns between them
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      zg += __shfl_xor_sync(0xffffffffu, zg, o);
      zg8 += __shfl_xor_sync(0xffffffffu, zg8, o);
    }
    // thread t == 0 writes row g, thread t == 1 row g + 8
    const float z = (t == 0 ? zg : zg8) + b3;
    const int rr = t == 0 ? g : g + 8;
    // sigmoid by the hardware reciprocal and exponential (omega needs ~1e-3)
    if (t < 2 && rr < rows)
      omega[r0 + rr] =
          fmaxf(omega_max * rcp_approx(1.0f + ex2_approx(z * -1.44269504f)), OMEGA_MIN);
  }
}

// Gradient of sum_i domega_i * omega_i with respect to the parameters.
// Each chunk of BW_ROWS rows: thread r computes row r's activations and
// backpropagated signals into shared memory; then every thread owns a set of
// parameters and adds their per-row terms in row order.  Per-block sums go to
// gpart[block][param].
__global__ void __launch_bounds__(BW_ROWS)
    k_mlp_backward(int64_t n, const float* __restrict__ params, const float* __restrict__ feat,
                   float omega_max, const float* __restrict__ domega,
                   double* __restrict__ gpart) {
  __shared__ float p[NPARAM];
  __shared__ float sf[BW_ROWS][NF], sh1[BW_ROWS][NH], sh2[BW_ROWS][NH], sdu1[BW_ROWS][NH],
      sdu2[BW_ROWS][NH], sdz[BW_ROWS];
  for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) p[k] = params[k];
  constexpr int PER = (NPARAM + BW_ROWS - 1) / BW_ROWS;
  double acc[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) acc[q] = 0.0;
  __syncthreads();
  const int64_t nchunks = (n + BW_ROWS - 1) / BW_ROWS;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int r = threadIdx.x;
    const int64_t i = c * BW_ROWS + r;
    if (i < n) {
      float f[NF];
#pragma unroll
      for (int k = 0; k < NF; ++k) f[k] = sf[r][k] = feat[i * NF + k];
      RowAct a;
      mlp_row(p, f, a);
      const float ws = omega_max * a.sg;  // d omega / dz = omega_max s (1 - s) above the floor
      const float dz = ws > OMEGA_MIN ? domega[i] * ws * (1.0f - a.sg) : 0.0f;
      sdz[r] = dz;
      float dh1[NH];
#pragma unroll
      for (int k = 0; k < NH; ++k) dh1[k] = 0.0f;
      for (int o = 0; o < NH; ++o) {
        const float du2 = dz * p[OFF_W3 + o] * gelu_df(a.u2[o]);
        sdu2[r][o] = du2;
        sh2[r][o] = a.h2[o];
        sh1[r][o] = a.h1[o];
#pragma unroll 8
        for (int k = 0; k < NH; ++k) dh1[k] = fmaf(p[OFF_W2 + o * NH + k], du2, dh1[k]);
      }
      for (int o = 0; o < NH; ++o) sdu1[r][o] = dh1[o] * gelu_df(a.u1[o]);
    } else {
      sdz[r] = 0.0f;
      for (int k = 0; k < NF; ++k) sf[r][k] = 0.0f;
      for (int o = 0; o < NH; ++o) sdu1[r][o] = sdu2[r][o] = sh1[r][o] = sh2[r][o] = 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int k = threadIdx.x + q * BW_ROWS;
      if (k >= NPARAM) break;
      double s = 0.0;
      for (int rr = 0; rr < BW_ROWS; ++rr) {
        float t;
        if (k < OFF_B1) t = sdu1[rr][k / NF] * sf[rr][k % NF];
        else if (k < OFF_W2) t = sdu1[rr][k - OFF_B1];
        else if (k < OFF_B2) t = sdu2[rr][(k - OFF_W2) / NH] * sh1[rr][(k - OFF_W2) % NH];
        else if (k < OFF_W3) t = sdu2[rr][k - OFF_B2];
        else if (k < OFF_B3) t = sdz[rr] * sh2[rr][k - OFF_W3];
        else t = sdz[rr];
        s += (double)t;
      }
      acc[q] += s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int k = threadIdx.x + q * BW_ROWS;
    if (k < NPARAM) gpart[(int64_t)blockIdx.x * NPARAM + k] = acc[q];
  }
}

// grad (+)= sum over blocks of gpart, in block order.
__global__ void k_mlp_grad_reduce(int nblocks, const double* __restrict__ gpart, double* grad,
                                  int accumulate) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NPARAM; k += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += gpart[(int64_t)b * NPARAM + k];
    grad[k] = accumulate ? grad[k] + s : s;
  }
}

// Adam (Kingma & Ba 2015) on FP32 parameters with FP64 moments; clears grad.
__global__ void k_adam(float* params, double* grad, double* m, double* v, int t, double lr,
                       double b1, double b2, double eps, double scale) {
  const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NPARAM; k += gridDim.x * blockDim.x) {
    const double g = grad[k] * scale;
    m[k] = b1 * m[k] + (1.0 - b1) * g;
    v[k] = b2 * v[k] + (1.0 - b2) * g * g;
    params[k] = (float)((double)params[k] - lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps));
    grad[k] = 0.0;
  }
}

// Host-side initial weights: N(0, 1/fan_in) from splitmix64 (Steele, Lea,
// Flood 2014) with the Box-Muller transform; biases zero, output bias 4
// (omega ~ 0.98 at start, next to plain l1-Jacobi's omega = 1, so training
// moves away from the fallback only where the loss improves).
static void init_params(uint64_t seed, std::vector<float>& p) {
  p.assign(NPARAM, 0.0f);
  uint64_t state = seed;
  auto next = [&]() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto normal = [&]() {
    const double u1 = (double)(next() >> 11) * (1.0 / 9007199254740992.0);
    const double u2 = (double)(next() >> 11) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log1p(-u1)) * cos(6.283185307179586 * u2);
  };
  for (int k = 0; k < NH * NF; ++k) p[OFF_W1 + k] = (float)(normal() / sqrt((double)NF));
  for (int k = 0; k < NH * NH; ++k) p[OFF_W2 + k] = (float)(normal() / sqrt((double)NH));
  for (int k = 0; k < NH; ++k) p[OFF_W3 + k] = (float)(normal() / sqrt((double)NH));
  p[OFF_B3] = 4.0f;
}

}  // namespace amg

using namespace amg;

extern "C" {

int mlp_num_params(void) { return NPARAM; }

int mlp_create(uint64_t seed, mlp_handle** M) {
  if (!M) return AMG_ERR_ARG;
  *M = nullptr;
  mlp_handle* h = new mlp_handle();
  auto fail = [&](int rc) {
    h->arena.release_all();
    delete h;
    return rc;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(AMG_ERR_CUDA);
  // the forward pass loops over tiles in a grid of exactly the CTAs that fit
  // the GPU at once (a second, partial wave would double its tail)
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, amg::k_mlp_forward_tc,
                                                    amg::TC_WARPS * 32, 0) != cudaSuccess)
    return fail(AMG_ERR_CUDA);
  h->tc_blocks = h->num_sms * std::max(occ, 1);
  int rc;
  if ((rc = h->arena.alloc_n(&h->params, NPARAM)) < 0) return fail(rc);
  if ((rc = h->arena.alloc_n(&h->grad, NPARAM)) < 0) return fail(rc);
  if ((rc = h->arena.alloc_n(&h->m, NPARAM)) < 0) return fail(rc);
  if ((rc = h->arena.alloc_n(&h->v, NPARAM)) < 0) return fail(rc);
  if ((rc = h->arena.alloc_n(&h->gpart, (int64_t)BW_BLOCKS_MAX * NPARAM)) < 0) return fail(rc);
  std::vector<float> p;
  init_params(seed, p);
  if (cudaMemcpy(h->params, p.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(h->grad, 0, sizeof(double) * NPARAM) != cudaSuccess ||
      cudaMemset(h->m, 0, sizeof(double) * NPARAM) != cudaSuccess ||
      cudaMemset(h->v, 0, sizeof(double) * NPARAM) != cudaSuccess)
    return fail(AMG_ERR_CUDA);
  *M = h;
  return AMG_OK;
}

int mlp_destroy(mlp_handle* M) {
  if (M) {
    M->arena.release_all();
    delete M;
  }
  return AMG_OK;
}

int mlp_get_params(const mlp_handle* M, float* host) {
  if (!M || !host) return AMG_ERR_ARG;
  AMG_CUDA_TRY(cudaMemcpy(host, M->params, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost));
  return AMG_OK;
}

int mlp_set_params(mlp_handle* M, const float* host) {
  if (!M || !host) return AMG_ERR_ARG;
  AMG_CUDA_TRY(cudaMemcpy(M->params, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice));
  AMG_CUDA_TRY(cudaMemset(M->grad, 0, sizeof(double) * NPARAM));
  AMG_CUDA_TRY(cudaMemset(M->m, 0, sizeof(double) * NPARAM));
  AMG_CUDA_TRY(cudaMemset(M->v, 0, sizeof(double) * NPARAM));
  M->t = 0;
  return AMG_OK;
}

int mlp_set_exact_forward(mlp_handle* M, int exact) {
  if (!M || (exact != 0 && exact != 1)) return AMG_ERR_ARG;
  M->exact = exact;
  return AMG_OK;
}

int mlp_set_omega_max(mlp_handle* M, double omega_max) {
  if (!M || !(omega_max >= 1.0 && omega_max < 2.0)) return AMG_ERR_ARG;
  M->omega_max = (float)omega_max;
  return AMG_OK;
}

int mlp_get_grad(const mlp_handle* M, double* host) {
  if (!M || !host) return AMG_ERR_ARG;
  AMG_CUDA_TRY(cudaMemcpy(host, M->grad, sizeof(double) * NPARAM, cudaMemcpyDeviceToHost));
  return AMG_OK;
}

int mlp_features(const amg_csr* A, int64_t nx, int64_t ny, int64_t nz, float* feat,
                 amg_stream_t stream) {
  if (!A || !feat || nx < 1 || ny < 1 || nz < 1 || A->n != nx * ny * nz) return AMG_ERR_ARG;
  int dev = 0, sms = 0;
  AMG_CUDA_TRY(cudaGetDevice(&dev));
  AMG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int occ = 0;  // a grid of the CTAs that fit at once (no partial second wave)
  AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_features, 256, 0));
  k_features<<<grid_for(A->n, 256, sms, std::max(occ, 1)), 256, 0, (cudaStream_t)stream>>>(
      A->n, nx, nx * ny, A->rowptr, A->col, A->val, feat);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

int mlp_forward(const mlp_handle* M, int64_t n, const float* feat, float* omega,
                amg_stream_t stream) {
  if (!M || n < 0 || !feat || !omega) return AMG_ERR_ARG;
  if (n == 0) return AMG_OK;
  if (M->exact) {
    // FP32 CUDA-core pass; 5 blocks fit an SM (41.6 KB of shared memory each)
    k_mlp_forward_tiled<<<grid_for((n + 31) / 32, FW_WARPS, M->num_sms, 5), FW_WARPS * 32, 0,
                          (cudaStream_t)stream>>>(n, M->params, feat, M->omega_max, omega);
  } else {
    const int64_t tiles = (n + 15) / 16;
    const int grid = (int)std::min<int64_t>((tiles + TC_WARPS - 1) / TC_WARPS, M->tc_blocks);
    k_mlp_forward_tc<<<grid, TC_WARPS * 32, 0, (cudaStream_t)stream>>>(n, M->params, feat,
                                                                    M->omega_max, omega);
  }
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

__global__ void k_gelu_fast(int64_t n, const float* u, float* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = gelu_fast(u[i]);
}

int mlp_debug_gelu(const float* u, float* out, int64_t n, amg_stream_t stream) {
  if (!u || !out || n < 0) return AMG_ERR_ARG;
  if (n == 0) return AMG_OK;
  k_gelu_fast<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0,
                (cudaStream_t)stream>>>(n, u, out);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

int mlp_backward(mlp_handle* M, int64_t n, const float* feat, const float* domega,
                 int accumulate, amg_stream_t stream) {
  if (!M || n < 0 || !feat || !domega) return AMG_ERR_ARG;
  const int64_t chunks = (n + BW_ROWS - 1) / BW_ROWS;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, BW_BLOCKS_MAX));
  cudaStream_t s = (cudaStream_t)stream;
  k_mlp_backward<<<nb, BW_ROWS, 0, s>>>(n, M->params, feat, M->omega_max, domega, M->gpart);
  AMG_LAUNCH_CHECK();
  k_mlp_grad_reduce<<<(NPARAM + 255) / 256, 256, 0, s>>>(nb, M->gpart, M->grad, accumulate);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

int mlp_adam_step(mlp_handle* M, double lr, double beta1, double beta2, double eps,
                  double grad_scale, amg_stream_t stream) {
  if (!M || !(lr > 0.0)) return AMG_ERR_ARG;
  M->t += 1;
  k_adam<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      M->params, M->grad, M->m, M->v, M->t, lr, beta1, beta2, eps, grad_scale);
  AMG_LAUNCH_CHECK();
  return AMG_OK;
}

}  // extern "C"
