// CPU ORACLE (test infrastructure only) for the learned smoother weights.
//
// A small MLP maps nine per-row stencil features to a damping weight
// omega_i in (0, omega_max] (omega_max 1 by default, at most below 2) for the
// l1-Jacobi smoother, s_i = omega_i / d_i
// (Sec. 2.3, l1-Jacobi; the network itself is not in the paper).  Plain FP64
// statements of: the features, the forward pass, its gradient by the chain
// rule, an Adam step, and the two-grid loss
//     L = mean_j  log(||E^K e0_j||_A / ||e0_j||_A) / K,
//     E = S (I - P A_c^-1 P^T A) S,   S = I - diag(s) A,
// with its gradient with respect to omega by the adjoint (reverse) pass.
//
// Readings (listed in the design notes): features are the six neighbour
// coefficients a_ij / a_ii in the order -x, +x, -y, +y, -z, +z of a
// lexicographic grid (0 where absent), the l1 ratio sum_{j!=i}|a_ij| / a_ii,
// log(max|a_ij| / min|a_ij|) over present neighbours and the neighbour count
// / 6; GELU is the exact erf form; omega = max(omega_max sigmoid(z), 1e-3).
// Parameter layout (1409 values): W1[32][9], b1[32], W2[32][32], b2[32],
// W3[32], b3.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

constexpr int NF = 9, NH = 32;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NF, OFF_W2 = OFF_B1 + NH,
              OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH,
              NPARAM = OFF_B3 + 1;
constexpr double OMEGA_MIN = 1e-3;

double gelu(double u) { return 0.5 * u * (1.0 + std::erf(u / std::sqrt(2.0))); }
double gelu_d(double u) {
  const double pdf = std::exp(-0.5 * u * u) / std::sqrt(2.0 * M_PI);
  return 0.5 * (1.0 + std::erf(u / std::sqrt(2.0))) + u * pdf;
}
double sigmoid(double z) { return 1.0 / (1.0 + std::exp(-z)); }

struct Act {
  double u1[NH], h1[NH], u2[NH], h2[NH], z, sg, omega;
};

// omega = max(omega_max * sigmoid(z), OMEGA_MIN): omega_max = 1 is the
// configuration's clamp to (0, 1]; omega_max in (1, 2) lets the network
// over-relax while 2 diag(d / omega) - A stays positive definite (d the l1
// row sums, so diag(d) - A is diagonally dominant): the smoother stays
// A-convergent and the V-cycle SPD.
void forward_row(const double* p, const double* f, Act& a, double omega_max) {
  for (int o = 0; o < NH; ++o) {
    double s = p[OFF_B1 + o];
    for (int i = 0; i < NF; ++i) s += p[OFF_W1 + o * NF + i] * f[i];
    a.u1[o] = s;
    a.h1[o] = gelu(s);
  }
  for (int o = 0; o < NH; ++o) {
    double s = p[OFF_B2 + o];
    for (int i = 0; i < NH; ++i) s += p[OFF_W2 + o * NH + i] * a.h1[i];
    a.u2[o] = s;
    a.h2[o] = gelu(s);
  }
  double z = p[OFF_B3];
  for (int i = 0; i < NH; ++i) z += p[OFF_W3 + i] * a.h2[i];
  a.z = z;
  a.sg = sigmoid(z);
  a.omega = std::max(omega_max * a.sg, OMEGA_MIN);
}

// Adds d(omega)/d(params) * g to grad (d omega / dz = omega_max s (1 - s)
// above the floor, 0 on it).
void backward_row(const double* p, const double* f, const Act& a, double g, double* grad,
                  double omega_max) {
  const double ws = omega_max * a.sg;
  const double dz = ws > OMEGA_MIN ? g * ws * (1.0 - a.sg) : 0.0;
  grad[OFF_B3] += dz;
  double du2[NH];
  for (int i = 0; i < NH; ++i) {
    grad[OFF_W3 + i] += dz * a.h2[i];
    du2[i] = dz * p[OFF_W3 + i] * gelu_d(a.u2[i]);
  }
  double dh1[NH] = {0};
  for (int o = 0; o < NH; ++o) {
    grad[OFF_B2 + o] += du2[o];
    for (int i = 0; i < NH; ++i) {
      grad[OFF_W2 + o * NH + i] += du2[o] * a.h1[i];
      dh1[i] += p[OFF_W2 + o * NH + i] * du2[o];
    }
  }
  for (int o = 0; o < NH; ++o) {
    const double du1 = dh1[o] * gelu_d(a.u1[o]);
    grad[OFF_B1 + o] += du1;
    for (int i = 0; i < NF; ++i) grad[OFF_W1 + o * NF + i] += du1 * f[i];
  }
}

// ---------------------------------------------------------------- two-grid

struct Csr {
  int64_t n;
  const int64_t* rp;
  const int32_t* ci;
  const double* v;
};

void spmv(const Csr& A, const double* x, double* y) {
  for (int64_t i = 0; i < A.n; ++i) {
    double s = 0.0;
    for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) s += A.v[e] * x[A.ci[e]];
    y[i] = s;
  }
}

double dot(int64_t n, const double* x, const double* y) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

// Exact coarse solve y = A_c^-1 g by dense Cholesky of A_c (n_c small).
struct Dense {
  int64_t n;
  std::vector<double> L;
  bool init(const Csr& A) {
    n = A.n;
    std::vector<double> a(n * n, 0.0);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t e = A.rp[i]; e < A.rp[i + 1]; ++e) a[i * n + A.ci[e]] = A.v[e];
    L.assign(n * n, 0.0);
    for (int64_t k = 0; k < n; ++k) {
      if (!(a[k * n + k] > 0.0)) return false;
      const double lkk = std::sqrt(a[k * n + k]);
      L[k * n + k] = lkk;
      for (int64_t i = k + 1; i < n; ++i) L[i * n + k] = a[i * n + k] / lkk;
      for (int64_t j = k + 1; j < n; ++j)
        for (int64_t i = j; i < n; ++i) a[i * n + j] -= L[i * n + k] * L[j * n + k];
    }
    return true;
  }
  void solve(const double* b, double* x) const {
    std::vector<double> y(n);
    for (int64_t i = 0; i < n; ++i) {
      double s = b[i];
      for (int64_t k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
      y[i] = s / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int64_t k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
      x[i] = s / L[i * n + i];
    }
  }
};

}  // namespace

extern "C" {

int mlp_orc_nparam() { return NPARAM; }

// Nine features per row of a 7-point operator on an nx x ny x nz grid.
void mlp_orc_features(int64_t nx, int64_t ny, int64_t nz, const int64_t* rp, const int32_t* ci,
                      const double* v, double* feat) {
  const int64_t n = nx * ny * nz;
  for (int64_t i = 0; i < n; ++i) {
    double aii = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
      if (ci[e] == i) aii = v[e];
    double off[6] = {0, 0, 0, 0, 0, 0}, l1 = 0.0, amax = 0.0, amin = 0.0;
    int cnt = 0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int64_t d = (int64_t)ci[e] - i;
      if (d == 0) continue;
      int slot = -1;
      if (d == -1) slot = 0;
      else if (d == 1) slot = 1;
      else if (d == -nx) slot = 2;
      else if (d == nx) slot = 3;
      else if (d == -nx * ny) slot = 4;
      else if (d == nx * ny) slot = 5;
      if (slot >= 0) off[slot] = v[e] / aii;
      const double m = std::fabs(v[e]);
      l1 += m;
      amax = cnt == 0 ? m : std::max(amax, m);
      amin = cnt == 0 ? m : std::min(amin, m);
      ++cnt;
    }
    double* f = feat + i * NF;
    for (int k = 0; k < 6; ++k) f[k] = off[k];
    f[6] = l1 / aii;
    f[7] = (cnt > 0 && amin > 0.0) ? std::log(amax / amin) : 0.0;
    f[8] = cnt / 6.0;
  }
}

void mlp_orc_forward(int64_t n, const double* params, const double* feat, double omega_max,
                     double* omega, double* z) {
  Act a;
  for (int64_t i = 0; i < n; ++i) {
    forward_row(params, feat + i * NF, a, omega_max);
    omega[i] = a.omega;
    if (z) z[i] = a.z;
  }
}

// grad = sum_i domega_i * d omega_i / d params.
void mlp_orc_backward(int64_t n, const double* params, const double* feat, double omega_max,
                      const double* domega, double* grad) {
  std::fill(grad, grad + NPARAM, 0.0);
  Act a;
  for (int64_t i = 0; i < n; ++i) {
    forward_row(params, feat + i * NF, a, omega_max);
    backward_row(params, feat + i * NF, a, domega[i], grad, omega_max);
  }
}

// One Adam step (Kingma & Ba 2015) at step t >= 1 on all parameters.
void mlp_orc_adam(int np, double* params, const double* grad, double* m, double* v, int t,
                  double lr, double b1, double b2, double eps) {
  const double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
  for (int k = 0; k < np; ++k) {
    m[k] = b1 * m[k] + (1.0 - b1) * grad[k];
    v[k] = b2 * v[k] + (1.0 - b2) * grad[k] * grad[k];
    params[k] -= lr * (m[k] / c1) / (std::sqrt(v[k] / c2) + eps);
  }
}

// Two-grid loss and its gradient with respect to omega.  A: fine matrix;
// agg: row -> aggregate (0/1 P); Ac: Galerkin matrix P^T A P; omega: damping
// weights (s_i = omega_i / d_i, d_i = sum_j |a_ij|); e0: nsamples x n initial
// errors (row-major by sample).  Returns 0, or -1 if A_c is not SPD.
int tg_orc_loss(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                const int32_t* agg, int64_t nc, const int64_t* rpc, const int32_t* cic,
                const double* vc, const double* omega, int nsamples, int K, const double* e0,
                double* loss, double* domega) {
  const Csr A{n, rp, ci, v}, Ac{nc, rpc, cic, vc};
  Dense coarse;
  if (!coarse.init(Ac)) return -1;
  std::vector<double> d(n), s(n), sbar(n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    double t = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) t += std::fabs(v[e]);
    d[i] = t;
    s[i] = omega[i] / t;
  }
  // C x = x - P A_c^-1 P^T A x ;  C^T x = x - A P A_c^-1 P^T x
  std::vector<double> g(nc), y(nc), tmp(n), tmp2(n);
  auto coarse_fwd = [&](const double* x, double* out) {
    spmv(A, x, tmp.data());
    std::fill(g.begin(), g.end(), 0.0);
    for (int64_t i = 0; i < n; ++i) g[agg[i]] += tmp[i];
    coarse.solve(g.data(), y.data());
    for (int64_t i = 0; i < n; ++i) out[i] = x[i] - y[agg[i]];
  };
  auto coarse_adj = [&](const double* x, double* out) {
    std::fill(g.begin(), g.end(), 0.0);
    for (int64_t i = 0; i < n; ++i) g[agg[i]] += x[i];
    coarse.solve(g.data(), y.data());
    for (int64_t i = 0; i < n; ++i) tmp2[i] = y[agg[i]];
    spmv(A, tmp2.data(), tmp.data());
    for (int64_t i = 0; i < n; ++i) out[i] = x[i] - tmp[i];
  };
  auto smooth_adj = [&](const double* x, double* out) {  // S^T x = x - A (s o x)
    for (int64_t i = 0; i < n; ++i) tmp2[i] = s[i] * x[i];
    spmv(A, tmp2.data(), tmp.data());
    for (int64_t i = 0; i < n; ++i) out[i] = x[i] - tmp[i];
  };
  double total = 0.0;
  std::vector<std::vector<double>> Ae(K, std::vector<double>(n)), Ac_(K, std::vector<double>(n));
  std::vector<double> e(n), a(n), c(n), Ax(n), eb(n), cb(n), ab(n);
  for (int j = 0; j < nsamples; ++j) {
    std::memcpy(e.data(), e0 + (int64_t)j * n, sizeof(double) * n);
    spmv(A, e.data(), Ax.data());
    const double n0 = dot(n, e.data(), Ax.data());
    for (int k = 0; k < K; ++k) {
      spmv(A, e.data(), Ae[k].data());
      for (int64_t i = 0; i < n; ++i) a[i] = e[i] - s[i] * Ae[k][i];  // pre-smooth
      coarse_fwd(a.data(), c.data());                                  // coarse correction
      spmv(A, c.data(), Ac_[k].data());
      for (int64_t i = 0; i < n; ++i) e[i] = c[i] - s[i] * Ac_[k][i];  // post-smooth
    }
    spmv(A, e.data(), Ax.data());
    const double nK = dot(n, e.data(), Ax.data());
    total += 0.5 * std::log(nK / n0) / K;
    // reverse pass: d/de_K of log(sqrt(e^T A e)) / K / nsamples
    for (int64_t i = 0; i < n; ++i) eb[i] = Ax[i] / (nK * K * nsamples);
    for (int k = K - 1; k >= 0; --k) {
      for (int64_t i = 0; i < n; ++i) sbar[i] -= eb[i] * Ac_[k][i];
      smooth_adj(eb.data(), cb.data());
      coarse_adj(cb.data(), ab.data());
      for (int64_t i = 0; i < n; ++i) sbar[i] -= ab[i] * Ae[k][i];
      smooth_adj(ab.data(), eb.data());
    }
  }
  *loss = total / nsamples;
  if (domega)
    for (int64_t i = 0; i < n; ++i) domega[i] = sbar[i] / d[i];
  return 0;
}

}  // extern "C"
