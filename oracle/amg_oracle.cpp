// CPU ORACLE -- test infrastructure only.
//
// A plain, slow, FP64 statement of what the solve path computes: CSR SpMV,
// the l1-Jacobi diagonal, compatible-weighted-matching edge weights, greedy
// (descending-key) maximum-weight matching, aggregate numbering, the Galerkin
// triple product, dense Cholesky, the V(1,1) cycle of Eq. (amg) and PCG.
// Only the tests, the smoke check and the benchmark's CPU-baseline leg may
// load this library; the GPU library never links or calls it, and this file
// shares no code with it.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared (see build.py).
// -ffp-contract=off keeps every a*b+c as two roundings, so the setup values
// (weights, Galerkin sums, l1 diagonal) are reproducible bit for bit.
//
// Readings of the paper used here (each also listed in the design notes):
//  * Matching weight (Sec. 2.3, "Coupled Aggregation Based on Compatible
//    Weighted Matching"; the paper names the edge weight matrix C without
//    defining it).  From the compatible-weighted-matching method it cites:
//      c_ij = 1 - 2 a_ij w_i w_j / (a_ii w_i^2 + a_jj w_j^2),
//    evaluated as num = ((2*a_ij)*w_i)*w_j, den = (a_ii*w_i)*w_i +
//    (a_jj*w_j)*w_j, c = 1 - num/den, using the entry stored in row
//    min(i, j).  Only edges with c > 0 may be matched.
//  * Approximate maximum-weight matching: edges ordered by the strict key
//    (c, -min, -max), larger first (equal weights go to the edge with the
//    smaller endpoints, the order a sequential greedy pass over the rows
//    takes); matched greedily in descending key order, which is the unique
//    result of locally-dominant matching under a strict total order.
//  * k matching sweeps give aggregates of at most 2^k rows (Sec. 2.3); sweep
//    s+1 matches the Galerkin matrix of the composite map after sweep s.
//    Aggregates are numbered in the order of their smallest member.
//  * P is piecewise constant with 0/1 entries (the paper's columns are
//    normalised; a diagonal rescaling of P leaves the V-cycle unchanged).
//  * Galerkin sum (A_c)_IJ = sum of a_ij over agg(i)=I, agg(j)=J taken in
//    ascending (min(i,j), max(i,j), [i>j]) order, which makes A_c bitwise
//    symmetric whenever A is.
//  * l1 diagonal (Sec. 2.3, l1-Jacobi): d_i = sum_j |a_ij| in ascending
//    column order (a_ii > 0); the smoother scale is s_i = w_i * (1.0 / d_i)
//    with w_i the damping weight (1 for plain l1-Jacobi).
//  * Coarsening stops when n_l <= max_coarse, when n_{l+1} > 0.9 n_l, or at
//    max_levels levels; the coarsest level is solved by dense Cholesky.
//  * Smoother sweeps (Sec. 3, the VBM/SMATCH/VMATCH configurations): nu
//    l1-Jacobi sweeps before and nu after the coarse correction, the first
//    pre-sweep from a zero guess.  The variable V-cycle (VMATCH) uses nu_0
//    sweeps on level 0, doubled on each coarser level: nu_l = nu_0 * 2^l.
//  * Smoothed prolongator (Sec. 2.3, SMATCH): P = (I - w D^-1 A) P_hat with
//    D = diag(A) and w = 1 / ||D^-1 A||_inf = 1 / max_i (sum_j |a_ij|) / a_ii.
//    Entry (i, J) of P is [agg(i) = J] - w * ((A P_hat)_iJ / a_ii), where
//    (A P_hat)_iJ sums a_ij over agg(j) = J in ascending j; P's columns are
//    kept ascending.  The coarse matrix is P^T (A P) by two sparse products;
//    each output entry sums its contributions in ascending order of the
//    inner index, each as one product and one addition (no fused multiply-
//    add).  The V-cycle restricts with P^T and prolongs with P.
//  * Filtered prolongator smoothing (an option, off by default; the paper's
//    formula uses A itself): with a threshold theta_f > 0 the smoothing uses
//    A_F, which keeps the diagonal and the entries with |a_ij| >=
//    theta_f * sqrt(a_ii * a_jj) (the entry of row i) and adds the dropped
//    entries of each row, in stored order, to its diagonal (row sums kept):
//    P = P_hat - w D^-1 (A_F P_hat), with D = diag(A) and w = 1 / ||D^-1 A||_inf
//    as the paper defines them (a row whose couplings are all weak then keeps
//    its P_hat row instead of dividing by a vanishing filtered diagonal); the
//    coarse matrix is still P^T (A P) with the unfiltered A.
//  * Decoupled Vanek-Mandel-Brezina aggregation (Sec. 2.3, VBM), on one
//    process, so "decoupled" changes nothing.  Strong neighbourhood
//    N_i = {i} + {j != i : |a_ij| >= theta * sqrt(a_ii * a_jj)}, the value of
//    edge {i, j} read from row min(i, j) (as for the matching weights; an edge
//    missing from that row is not strong).  Phase 1: rows in ascending order;
//    a row whose whole N_i is unaggregated starts the aggregate N_i.
//    Phase 2 ("remaining nodes are added to the nearest aggregates"): every
//    row left joins the phase-1 aggregate of its strong neighbour with the
//    largest |a_ij| (the smaller j on ties).  Phase 3: rows still left, in
//    ascending order, start an aggregate with their unaggregated strong
//    neighbours (empty when the pattern is symmetric: a row outside every
//    phase-1 aggregate shares a strong neighbour with one).  Aggregates are
//    numbered as they are created; P_hat has w = 1 (the constant near-kernel
//    vector).  The paper leaves theta to the user; the default is 0.01.
//  * Iterative coarsest solve (VBM, Sec. 3): PCG with the coarsest level's
//    l1-Jacobi scaling as preconditioner, zero initial guess, at most maxit
//    iterations; it stops once ||r|| <= tol * ||b|| (the paper gives only the
//    iteration cap; the tolerance is a parameter), and on p^T A p <= 0.
//  * Dot products: partial sums over fixed blocks of 4096 entries, then the
//    partials in order.
//
// Threads.  Built plainly this is a single-thread program.  Built with
// -fopenmp (liboracle_omp.so, for timing the CPU baseline on all host cores)
// the loops marked ROWS_PARALLEL run their iterations on several threads.
// Each such loop writes only its own row's (or aggregate's, or dot-product
// block's) output and reads nothing another iteration writes, and every sum
// keeps its order, so both builds give the same bits.  The setup phase stays
// serial.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#define ROWS_PARALLEL _Pragma("omp parallel for schedule(static)")
#else
#define ROWS_PARALLEL
#endif

namespace {

struct Csr {
  int64_t n = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  int64_t nnz() const { return (int64_t)col.size(); }
};

struct Level {
  Csr A;
  std::vector<double> dinv;      // smoother scale s_i
  std::vector<int32_t> agg;      // row -> aggregate on the next level
  std::vector<int32_t> members;  // nc x stride, ascending, -1 padded
  int stride = 0;  // 1 << sweeps (matching), or >= the largest aggregate (VBM)
  int64_t nc = 0;
  // smoothed prolongator (empty when P is the 0/1 aggregate map) and P^T
  Csr P, Pt;
  double wp = 0.0;  // its damping w = 1 / ||D^-1 A||_inf
};

struct Hierarchy {
  int sweeps = 2;
  int smooth_p = 0;  // 1: smoothed prolongators (Sec. 2.3)
  int aggregation = 0;  // 0: matching sweeps; 1: VBM with strength theta
  double theta = 0.01;
  double pfilter = 0.0;  // > 0: smooth P with the filtered matrix A_F
  std::vector<Level> lev;
  std::vector<double> chol;  // dense lower factor of the coarsest matrix, row-major
  int64_t nco = 0;
  // cycle: smoother sweeps nu_0, variable V-cycle (nu_l = nu_0 * 2^l), and the
  // coarsest solver (0 dense Cholesky, 1 PCG with l1-Jacobi)
  int nu0 = 1;
  int variable = 0;
  int coarse = 0;
  int coarse_maxit = 40;
  double coarse_tol = 1e-4;
};

// ---------------------------------------------------------------- basics

double dot_blocked(int64_t n, const double* x, const double* y) {
  const int64_t B = 4096;
  const int64_t nb = (n + B - 1) / B;
  std::vector<double> part(nb);
  ROWS_PARALLEL
  for (int64_t k = 0; k < nb; ++k) {
    const int64_t b0 = k * B, b1 = std::min(n, b0 + B);
    double s = 0.0;
    for (int64_t i = b0; i < b1; ++i) s += x[i] * y[i];
    part[k] = s;
  }
  double total = 0.0;
  for (int64_t k = 0; k < nb; ++k) total += part[k];
  return total;
}

void spmv(const Csr& A, const double* x, double* y) {
  ROWS_PARALLEL
  for (int64_t i = 0; i < A.n; ++i) {
    double s = 0.0;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) s += A.val[e] * x[A.col[e]];
    y[i] = s;
  }
}

double diag_of(const Csr& A, int64_t i) {
  for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e)
    if (A.col[e] == i) return A.val[e];
  return 0.0;
}

// splitmix64 finaliser (Steele, Lea, Flood 2014); exported only so the tests
// can pin the input generator's random stream against the published values.
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double match_weight(double aij, double aii, double ajj, double wi, double wj) {
  double num = ((2.0 * aij) * wi) * wj;
  double den = (aii * wi) * wi + (ajj * wj) * wj;
  return 1.0 - num / den;
}

// ---------------------------------------------------------------- matching

struct Edge {
  double c;
  int32_t lo, hi;
};

bool heavier(const Edge& a, const Edge& b) {
  if (a.c != b.c) return a.c > b.c;
  if (a.lo != b.lo) return a.lo < b.lo;
  return a.hi < b.hi;
}

// Greedy matching in descending key order; mate[i] = partner or -1.
void match_greedy(const Csr& A, const double* w, std::vector<int32_t>& mate) {
  const int64_t n = A.n;
  std::vector<double> d(n);
  for (int64_t i = 0; i < n; ++i) d[i] = diag_of(A, i);
  std::vector<Edge> edges;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      int64_t j = A.col[e];
      if (j <= i) continue;  // the edge is read from row min(i, j)
      double wi = w ? w[i] : 1.0, wj = w ? w[j] : 1.0;
      double c = match_weight(A.val[e], d[i], d[j], wi, wj);
      if (!(c > 0.0)) continue;
      Edge ed;
      ed.c = c;
      ed.lo = (int32_t)i;
      ed.hi = (int32_t)j;
      edges.push_back(ed);
    }
  }
  std::sort(edges.begin(), edges.end(), heavier);
  mate.assign(n, -1);
  for (const Edge& ed : edges) {
    if (mate[ed.lo] < 0 && mate[ed.hi] < 0) {
      mate[ed.lo] = ed.hi;
      mate[ed.hi] = ed.lo;
    }
  }
}

// ---------------------------------------------------------------- VBM

// Value of edge {i, j} (i != j): the entry of row min(i, j); false if absent.
bool edge_value(const Csr& A, int64_t i, int64_t j, double aij_row_i, double* out) {
  if (j > i) {
    *out = aij_row_i;
    return true;
  }
  for (int64_t e = A.rowptr[j]; e < A.rowptr[j + 1]; ++e)
    if (A.col[e] == i) {
      *out = A.val[e];
      return true;
    }
  return false;
}

// Decoupled VBM aggregation (see the header); returns the aggregate count.
int64_t vbm_aggregate(const Csr& A, double theta, std::vector<int32_t>& agg) {
  const int64_t n = A.n;
  std::vector<double> d(n);
  for (int64_t i = 0; i < n; ++i) d[i] = diag_of(A, i);
  // strong[e]: entry e of row i is a strong neighbour j != i
  std::vector<char> strong(A.col.size(), 0);
  std::vector<double> mag(A.col.size(), 0.0);  // |edge value|
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const int64_t j = A.col[e];
      double a;
      if (j == i || !edge_value(A, i, j, A.val[e], &a)) continue;
      mag[e] = std::fabs(a);
      strong[e] = mag[e] >= theta * std::sqrt(d[i] * d[j]);
    }
  agg.assign(n, -1);
  int64_t nc = 0;
  // phase 1
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool free = true;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1] && free; ++e)
      if (strong[e] && agg[A.col[e]] >= 0) free = false;
    if (!free) continue;
    agg[i] = (int32_t)nc;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e)
      if (strong[e]) agg[A.col[e]] = (int32_t)nc;
    ++nc;
  }
  // phase 2: against the phase-1 aggregates only
  const std::vector<int32_t> agg1 = agg;
  for (int64_t i = 0; i < n; ++i) {
    if (agg1[i] >= 0) continue;
    int64_t best = -1;
    double bm = 0.0;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const int64_t j = A.col[e];
      if (!strong[e] || agg1[j] < 0) continue;
      if (best < 0 || mag[e] > bm || (mag[e] == bm && j < best)) {
        best = j;
        bm = mag[e];
      }
    }
    if (best >= 0) agg[i] = agg1[best];
  }
  // phase 3
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    agg[i] = (int32_t)nc;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e)
      if (strong[e] && agg[A.col[e]] < 0) agg[A.col[e]] = (int32_t)nc;
    ++nc;
  }
  return nc;
}

// Smallest power of two >= the largest aggregate.
int member_stride(const std::vector<int32_t>& agg, int64_t nc) {
  std::vector<int> cnt(nc, 0);
  int m = 1;
  for (int32_t a : agg) m = std::max(m, ++cnt[a]);
  int s = 1;
  while (s < m) s <<= 1;
  return s;
}

// Aggregates numbered in the order of their smallest member.
int64_t number_pairs(const std::vector<int32_t>& mate, std::vector<int32_t>& agg) {
  const int64_t n = (int64_t)mate.size();
  agg.assign(n, -1);
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i) {
    int32_t m = mate[i];
    if (m < 0 || m > i) {
      agg[i] = (int32_t)nc;
      if (m >= 0) agg[m] = (int32_t)nc;
      ++nc;
    }
  }
  return nc;
}

// ---------------------------------------------------------------- Galerkin

struct Contrib {
  int32_t J;
  int64_t lo, hi;
  int flip;  // 1 when the fine entry is (hi, lo)
  double v;
};

bool contrib_less(const Contrib& a, const Contrib& b) {
  if (a.J != b.J) return a.J < b.J;
  if (a.lo != b.lo) return a.lo < b.lo;
  if (a.hi != b.hi) return a.hi < b.hi;
  return a.flip < b.flip;
}

void members_of(const std::vector<int32_t>& agg, int64_t nc, int stride,
                std::vector<int32_t>& mem) {
  mem.assign(nc * stride, -1);
  std::vector<int> cnt(nc, 0);
  for (int64_t i = 0; i < (int64_t)agg.size(); ++i) {
    int32_t I = agg[i];
    mem[(int64_t)I * stride + cnt[I]++] = (int32_t)i;
  }
}

// (A_c)_IJ = sum_{agg(i)=I, agg(j)=J} a_ij in canonical order.
void galerkin(const Csr& A, const std::vector<int32_t>& agg, int64_t nc,
              const std::vector<int32_t>& mem, int stride, Csr& Ac) {
  Ac.n = nc;
  Ac.rowptr.assign(nc + 1, 0);
  Ac.col.clear();
  Ac.val.clear();
  std::vector<Contrib> buf;
  for (int64_t I = 0; I < nc; ++I) {
    buf.clear();
    for (int s = 0; s < stride; ++s) {
      int32_t i = mem[I * stride + s];
      if (i < 0) break;
      for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
        int64_t j = A.col[e];
        Contrib c;
        c.J = agg[j];
        c.lo = std::min<int64_t>(i, j);
        c.hi = std::max<int64_t>(i, j);
        c.flip = i > j ? 1 : 0;
        c.v = A.val[e];
        buf.push_back(c);
      }
    }
    std::sort(buf.begin(), buf.end(), contrib_less);
    size_t k = 0;
    while (k < buf.size()) {
      int32_t J = buf[k].J;
      double s = buf[k].v;
      ++k;
      while (k < buf.size() && buf[k].J == J) {
        s = s + buf[k].v;
        ++k;
      }
      Ac.col.push_back(J);
      Ac.val.push_back(s);
    }
    Ac.rowptr[I + 1] = (int64_t)Ac.col.size();
  }
}

void l1_scale(const Csr& A, const double* omega, std::vector<double>& dinv) {
  dinv.resize(A.n);
  for (int64_t i = 0; i < A.n; ++i) {
    double d = 0.0;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) d += std::fabs(A.val[e]);
    double w = omega ? omega[i] : 1.0;
    dinv[i] = w * (1.0 / d);
  }
}

// ---------------------------------------------------------------- smoothed P

// w = 1 / max_i (sum_j |a_ij|) / a_ii.
double prolongator_damping(const Csr& A) {
  double m = 0.0;
  for (int64_t i = 0; i < A.n; ++i) {
    double s = 0.0, d = 0.0;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      s += std::fabs(A.val[e]);
      if (A.col[e] == i) d = A.val[e];
    }
    m = std::max(m, s / d);
  }
  return 1.0 / m;
}

// P = P_hat - w D^-1 (S P_hat), columns ascending; D = diag(A), S = A or its
// filtered form A_F.
void smoothed_prolongator(const Csr& A, const Csr& S, const std::vector<int32_t>& agg,
                          int64_t nc, double w, Csr& P) {
  P.n = A.n;
  P.rowptr.assign(A.n + 1, 0);
  P.col.clear();
  P.val.clear();
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t i = 0; i < A.n; ++i) {
    row.clear();
    double aii = 0.0;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e)
      if (A.col[e] == i) aii = A.val[e];
    for (int64_t e = S.rowptr[i]; e < S.rowptr[i + 1]; ++e) {
      const int32_t J = agg[S.col[e]];
      bool found = false;
      for (auto& c : row)
        if (c.first == J) {
          c.second = c.second + S.val[e];
          found = true;
        }
      if (!found) row.push_back({J, S.val[e]});
    }
    std::sort(row.begin(), row.end(),
              [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                return a.first < b.first;
              });
    for (const auto& c : row) {
      const double ind = c.first == agg[i] ? 1.0 : 0.0;
      P.col.push_back(c.first);
      P.val.push_back(ind - w * (c.second / aii));
    }
    P.rowptr[i + 1] = (int64_t)P.col.size();
  }
  (void)nc;
}

// C = X Y (X: n x m, Y: m x k CSR, columns ascending in each row): entry
// (i, J) sums x_ik * y_kJ over the entries k of row i in ascending order.
void spgemm(const Csr& X, const Csr& Y, Csr& Cm) {
  Cm.n = X.n;
  Cm.rowptr.assign(X.n + 1, 0);
  Cm.col.clear();
  Cm.val.clear();
  std::vector<std::pair<int32_t, double>> acc;  // (J, sum), first-touch order
  for (int64_t i = 0; i < X.n; ++i) {
    acc.clear();
    for (int64_t e = X.rowptr[i]; e < X.rowptr[i + 1]; ++e) {
      const int64_t k = X.col[e];
      for (int64_t f = Y.rowptr[k]; f < Y.rowptr[k + 1]; ++f) {
        const double t = X.val[e] * Y.val[f];
        bool found = false;
        for (auto& c : acc)
          if (c.first == Y.col[f]) {
            c.second = c.second + t;
            found = true;
            break;
          }
        if (!found) acc.push_back({Y.col[f], t});
      }
    }
    std::sort(acc.begin(), acc.end(),
              [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                return a.first < b.first;
              });
    for (const auto& c : acc) {
      Cm.col.push_back(c.first);
      Cm.val.push_back(c.second);
    }
    Cm.rowptr[i + 1] = (int64_t)Cm.col.size();
  }
}

Csr transpose(const Csr& X, int64_t ncols) {
  Csr T;
  T.n = ncols;
  T.rowptr.assign(ncols + 1, 0);
  for (int32_t c : X.col) ++T.rowptr[c + 1];
  for (int64_t J = 0; J < ncols; ++J) T.rowptr[J + 1] += T.rowptr[J];
  T.col.resize(X.col.size());
  T.val.resize(X.col.size());
  std::vector<int64_t> pos(T.rowptr.begin(), T.rowptr.end() - 1);
  for (int64_t i = 0; i < X.n; ++i)  // rows ascending: each column of T ascending
    for (int64_t e = X.rowptr[i]; e < X.rowptr[i + 1]; ++e) {
      const int64_t p = pos[X.col[e]]++;
      T.col[p] = (int32_t)i;
      T.val[p] = X.val[e];
    }
  return T;
}

// ---------------------------------------------------------------- Cholesky

// Right-looking Cholesky of a dense SPD n x n matrix (row-major, full).
// Returns 0, or -(k+1) when the k-th pivot is not positive.
int cholesky(int64_t n, std::vector<double> a, std::vector<double>& L) {
  L.assign(n * n, 0.0);
  for (int64_t k = 0; k < n; ++k) {
    double piv = a[k * n + k];
    if (!(piv > 0.0)) return -(int)(k + 1);
    double lkk = std::sqrt(piv);
    L[k * n + k] = lkk;
    for (int64_t i = k + 1; i < n; ++i) L[i * n + k] = a[i * n + k] / lkk;
    for (int64_t j = k + 1; j < n; ++j)
      for (int64_t i = j; i < n; ++i) a[i * n + j] -= L[i * n + k] * L[j * n + k];
  }
  return 0;
}

void chol_solve(int64_t n, const std::vector<double>& L, const double* b, double* x) {
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

std::vector<double> dense_of(const Csr& A) {
  std::vector<double> a(A.n * A.n, 0.0);
  for (int64_t i = 0; i < A.n; ++i)
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) a[i * A.n + A.col[e]] += A.val[e];
  return a;
}

// ---------------------------------------------------------------- hierarchy

Csr csr_copy(int64_t n, const int64_t* rp, const int32_t* ci, const double* v) {
  Csr A;
  A.n = n;
  A.rowptr.assign(rp, rp + n + 1);
  int64_t nnz = rp[n] - rp[0];
  A.col.assign(ci + rp[0], ci + rp[0] + nnz);
  A.val.assign(v + rp[0], v + rp[0] + nnz);
  if (rp[0] != 0)
    for (auto& p : A.rowptr) p -= rp[0];
  return A;
}

// A_F of the filtered prolongator smoothing (see the header).
Csr filtered_matrix(const Csr& A, double theta) {
  Csr F;
  F.n = A.n;
  F.rowptr.assign(A.n + 1, 0);
  std::vector<double> d(A.n);
  for (int64_t i = 0; i < A.n; ++i) d[i] = diag_of(A, i);
  for (int64_t i = 0; i < A.n; ++i) {
    double lump = 0.0;
    int64_t dpos = -1;
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const int64_t j = A.col[e];
      const double v = A.val[e];
      if (j == i) {
        dpos = (int64_t)F.col.size();
      } else if (!(std::fabs(v) >= theta * std::sqrt(d[i] * d[j]))) {
        lump = lump + v;
        continue;
      }
      F.col.push_back((int32_t)j);
      F.val.push_back(v);
    }
    if (dpos >= 0) F.val[dpos] = F.val[dpos] + lump;
    F.rowptr[i + 1] = (int64_t)F.col.size();
  }
  return F;
}

// The next level's matrix: P_hat^T A P_hat in canonical order, or with the
// smoothed prolongator P^T (A P) (which also keeps P and P^T on the level).
void coarse_matrix(const Hierarchy& H, Level& L, int stride, Csr& Ac) {
  if (!H.smooth_p) {
    galerkin(L.A, L.agg, L.nc, L.members, stride, Ac);
    return;
  }
  const Csr AF = H.pfilter > 0.0 ? filtered_matrix(L.A, H.pfilter) : Csr();
  L.wp = prolongator_damping(L.A);
  smoothed_prolongator(L.A, H.pfilter > 0.0 ? AF : L.A, L.agg, L.nc, L.wp, L.P);
  L.Pt = transpose(L.P, L.nc);
  Csr Q;
  spgemm(L.A, L.P, Q);
  spgemm(L.Pt, Q, Ac);
}

// Returns 0 or a negative status (-4 not SPD coarse matrix, -1 arguments).
// Largest diagonal block (system) of a level; the whole level without systems.
int64_t largest_block(const std::vector<int64_t>& sys, int64_t n) {
  if (sys.size() < 2) return n;
  int64_t m = 0;
  for (size_t k = 0; k + 1 < sys.size(); ++k) m = std::max(m, sys[k + 1] - sys[k]);
  return m;
}

// sys: first row of each of several independent systems stacked block
// diagonally (empty for one system).  With systems, coarsening stops once
// every system has at most max_coarse rows, so each keeps the coarsest level
// it would get alone; the coarsest matrix stays block diagonal.
// like: a hierarchy whose aggregates are reused level by level (new values,
// the same structure: Sec. 2.2 updates coefficients of a matrix whose
// structure is preserved and rebuilds on an assembled hierarchy); null to
// build the aggregates by matching.
int build(Hierarchy& H, Csr A0, int sweeps, int64_t max_coarse, int max_levels,
          double stall, int64_t max_dense, const double* omega,
          std::vector<int64_t> sys = std::vector<int64_t>(), const Hierarchy* like = nullptr,
          int smooth_p = 0, int aggregation = 0, double theta = 0.01, double pfilter = 0.0) {
  H.sweeps = sweeps;
  H.smooth_p = like ? like->smooth_p : smooth_p;
  H.aggregation = like ? like->aggregation : aggregation;
  H.theta = like ? like->theta : theta;
  H.pfilter = like ? like->pfilter : pfilter;
  H.lev.clear();
  H.lev.emplace_back();
  H.lev[0].A = std::move(A0);
  for (int l = 0;; ++l) {
    Level& L = H.lev[l];
    l1_scale(L.A, l == 0 ? omega : nullptr, L.dinv);
    const int64_t n = L.A.n;
    if (like) {
      if (l + 1 >= (int)like->lev.size()) break;
      L.agg = like->lev[l].agg;
      L.nc = like->lev[l].nc;
      L.members = like->lev[l].members;
      L.stride = like->lev[l].stride;
      Level next;
      coarse_matrix(H, L, L.stride, next.A);
      H.lev.push_back(std::move(next));
      continue;
    }
    if (largest_block(sys, n) <= max_coarse || l + 1 >= max_levels) break;
    std::vector<int32_t> comp(n);
    for (int64_t i = 0; i < n; ++i) comp[i] = (int32_t)i;
    int64_t nc = n;
    Csr Acur = L.A;  // sweep 1 matches A_l itself
    if (H.aggregation == 1) nc = vbm_aggregate(L.A, H.theta, comp);
    for (int s = 0; s < sweeps && H.aggregation == 0; ++s) {
      std::vector<int32_t> mate, ags;
      match_greedy(Acur, nullptr, mate);
      nc = number_pairs(mate, ags);
      for (int64_t i = 0; i < n; ++i) comp[i] = ags[comp[i]];
      if (s + 1 < sweeps) {
        std::vector<int32_t> mem;
        int st = 1 << (s + 1);
        members_of(comp, nc, st, mem);
        galerkin(L.A, comp, nc, mem, st, Acur);
      }
    }
    if ((double)nc > stall * (double)n) break;
    L.agg = comp;
    L.nc = nc;
    L.stride = H.aggregation == 1 ? member_stride(comp, nc) : 1 << sweeps;
    members_of(comp, nc, L.stride, L.members);
    Level next;
    coarse_matrix(H, L, L.stride, next.A);
    H.lev.push_back(std::move(next));
    if (sys.size() >= 2) {  // aggregates never span systems
      std::vector<int64_t> nxt(sys.size());
      for (size_t k = 0; k + 1 < sys.size(); ++k) nxt[k] = H.lev[l].agg[sys[k]];
      nxt.back() = nc;
      sys.swap(nxt);
    }
  }
  const Csr& C = H.lev.back().A;
  if (largest_block(sys, C.n) > max_dense) return -1;
  H.nco = C.n;
  return cholesky(C.n, dense_of(C), H.chol) == 0 ? 0 : -4;
}

// Coarsest solve by PCG with the l1-Jacobi preconditioner (see the header).
void coarse_pcg(const Hierarchy& H, const double* b, double* x) {
  const Level& L = H.lev.back();
  const int64_t n = L.A.n;
  std::vector<double> r(b, b + n), z(n), p(n), q(n);
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  const double bnorm = std::sqrt(dot_blocked(n, b, b));
  if (bnorm == 0.0) return;
  for (int64_t i = 0; i < n; ++i) z[i] = L.dinv[i] * r[i];
  p = z;
  double rz = dot_blocked(n, r.data(), z.data());
  for (int k = 0; k < H.coarse_maxit; ++k) {
    spmv(L.A, p.data(), q.data());
    const double pq = dot_blocked(n, p.data(), q.data());
    if (!(pq > 0.0)) break;
    const double alpha = rz / pq;
    for (int64_t i = 0; i < n; ++i) {
      x[i] = x[i] + alpha * p[i];
      r[i] = r[i] - alpha * q[i];
    }
    if (std::sqrt(dot_blocked(n, r.data(), r.data())) <= H.coarse_tol * bnorm) break;
    for (int64_t i = 0; i < n; ++i) z[i] = L.dinv[i] * r[i];
    const double rz_new = dot_blocked(n, r.data(), z.data());
    const double beta = rz_new / rz;
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rz = rz_new;
  }
}

// Smoother sweeps on level l.
int64_t sweeps_at(const Hierarchy& H, int l) {
  return H.variable ? (int64_t)H.nu0 << l : (int64_t)H.nu0;
}

// One l1-Jacobi sweep x <- x + S (b - A x); r is scratch.
void jacobi_sweep(const Level& L, const double* b, double* x, double* r) {
  const int64_t n = L.A.n;
  spmv(L.A, x, r);
  ROWS_PARALLEL
  for (int64_t i = 0; i < n; ++i) x[i] = x[i] + L.dinv[i] * (b[i] - r[i]);
}

// V(nu, nu) cycle with zero initial guess at every level (Eq. amg); nu = 1 is
// the V(1,1) cycle.
void vcycle(const Hierarchy& H, int l, const double* b, double* x) {
  const Level& L = H.lev[l];
  const int64_t n = L.A.n;
  if (l + 1 == (int)H.lev.size()) {
    if (H.coarse == 1)
      coarse_pcg(H, b, x);
    else
      chol_solve(n, H.chol, b, x);
    return;
  }
  const int64_t nu = sweeps_at(H, l);
  std::vector<double> r(n), bc(L.nc), xc(L.nc);
  ROWS_PARALLEL
  for (int64_t i = 0; i < n; ++i) x[i] = L.dinv[i] * b[i];  // pre-smooth, zero guess
  for (int64_t k = 1; k < nu; ++k) jacobi_sweep(L, b, x, r.data());
  spmv(L.A, x, r.data());
  ROWS_PARALLEL
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - r[i];  // residual
  const int stride = L.stride;
  if (H.smooth_p) {
    spmv(L.Pt, r.data(), bc.data());  // restriction b_c = P^T r
  } else {
    ROWS_PARALLEL
    for (int64_t I = 0; I < L.nc; ++I) {  // restriction b_c = P^T r
      double s = 0.0;
      for (int k = 0; k < stride; ++k) {
        int32_t i = L.members[I * stride + k];
        if (i < 0) break;
        s = (k == 0) ? r[i] : s + r[i];
      }
      bc[I] = s;
    }
  }
  vcycle(H, l + 1, bc.data(), xc.data());
  if (H.smooth_p) {  // prolongation x += P x_c
    spmv(L.P, xc.data(), r.data());
    ROWS_PARALLEL
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] + r[i];
  } else {
    ROWS_PARALLEL
    for (int64_t i = 0; i < n; ++i) x[i] = x[i] + xc[L.agg[i]];
  }
  for (int64_t k = 0; k < nu; ++k) jacobi_sweep(L, b, x, r.data());  // post-smooth
}

// ---------------------------------------------------------------- PCG

struct PcgOut {
  int iters = 0;
  int status = 0;  // 0 converged, 1 maxit, -2 breakdown, -3 nan
  double relres = 0, true_relres = 0;
};

PcgOut pcg(const Csr& A, const std::function<void(const double*, double*)>& prec,
           const double* b, double* x, double tol, int maxit, int beta_form,
           double* res_hist, double* x_hist) {
  const int64_t n = A.n;
  PcgOut o;
  std::vector<double> r(n), z(n), p(n), q(n), rold;
  spmv(A, x, q.data());
  ROWS_PARALLEL
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
  double bnorm = std::sqrt(dot_blocked(n, b, b));
  if (bnorm == 0.0) bnorm = 1.0;
  double rr = dot_blocked(n, r.data(), r.data());
  o.relres = std::sqrt(rr) / bnorm;
  if (res_hist) res_hist[0] = o.relres;
  if (x_hist) std::memcpy(x_hist, x, sizeof(double) * n);
  if (o.relres <= tol) return o;
  prec(r.data(), z.data());
  p = z;
  double rz = dot_blocked(n, r.data(), z.data());
  int k = 0;
  o.status = 1;
  for (; k < maxit; ++k) {
    spmv(A, p.data(), q.data());
    double pq = dot_blocked(n, p.data(), q.data());
    if (!(pq > 0.0)) {
      o.status = std::isnan(pq) ? -3 : -2;
      break;
    }
    double alpha = rz / pq;
    if (beta_form == 1) rold = r;
    ROWS_PARALLEL
    for (int64_t i = 0; i < n; ++i) {
      x[i] = x[i] + alpha * p[i];
      r[i] = r[i] - alpha * q[i];
    }
    rr = dot_blocked(n, r.data(), r.data());
    o.relres = std::sqrt(rr) / bnorm;
    if (res_hist) res_hist[k + 1] = o.relres;
    if (x_hist) std::memcpy(x_hist + (int64_t)(k + 1) * n, x, sizeof(double) * n);
    if (std::isnan(rr)) {
      o.status = -3;
      ++k;
      break;
    }
    if (o.relres <= tol) {
      o.status = 0;
      ++k;
      break;
    }
    prec(r.data(), z.data());
    double rz_new = dot_blocked(n, r.data(), z.data());
    double beta;
    if (beta_form == 1) {
      double zro = dot_blocked(n, z.data(), rold.data());
      beta = (rz_new - zro) / rz;
    } else {
      beta = rz_new / rz;
    }
    ROWS_PARALLEL
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rz = rz_new;
  }
  o.iters = k;
  spmv(A, x, q.data());
  ROWS_PARALLEL
  for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
  o.true_relres = std::sqrt(dot_blocked(n, q.data(), q.data())) / bnorm;
  return o;
}

}  // namespace

// ====================================================================== C-ABI
extern "C" {

double orc_dot(int64_t n, const double* x, const double* y) { return dot_blocked(n, x, y); }

// Threads the parallel row loops use (1 in the plain build).
int orc_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* x,
              double* y) {
  Csr A = csr_copy(n, rp, ci, v);
  spmv(A, x, y);
}

void orc_l1_scale(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                  const double* omega, double* dinv) {
  Csr A = csr_copy(n, rp, ci, v);
  std::vector<double> d;
  l1_scale(A, omega, d);
  std::memcpy(dinv, d.data(), sizeof(double) * n);
}

// Weight of every stored entry (0 on the diagonal), aligned with val.
void orc_match_weights(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                       const double* w, double* c) {
  Csr A = csr_copy(n, rp, ci, v);
  for (int64_t i = 0; i < n; ++i) {
    double aii = diag_of(A, i);
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      int64_t j = A.col[e];
      if (j == i) {
        c[e] = 0.0;
        continue;
      }
      int64_t e2 = (j < i) ? -1 : e;  // weight read from row min(i, j)
      double aij = A.val[e];
      if (e2 < 0)
        for (int64_t f = A.rowptr[j]; f < A.rowptr[j + 1]; ++f)
          if (A.col[f] == i) aij = A.val[f];
      c[e] = match_weight(aij, (j < i) ? diag_of(A, j) : aii, (j < i) ? aii : diag_of(A, j),
                          w ? w[std::min(i, j)] : 1.0, w ? w[std::max(i, j)] : 1.0);
    }
  }
}

uint64_t orc_mix64(uint64_t z) { return mix64(z); }

void orc_match(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* w,
               int32_t* mate) {
  Csr A = csr_copy(n, rp, ci, v);
  std::vector<int32_t> m;
  match_greedy(A, w, m);
  std::memcpy(mate, m.data(), sizeof(int32_t) * n);
}

int64_t orc_number_pairs(int64_t n, const int32_t* mate, int32_t* agg) {
  std::vector<int32_t> m(mate, mate + n), a;
  int64_t nc = number_pairs(m, a);
  std::memcpy(agg, a.data(), sizeof(int32_t) * n);
  return nc;
}

// Galerkin product into caller buffers.  Call with rp_c only to size it
// (col_c == nullptr), then again with col_c/val_c of rp_c[nc] entries.
void orc_galerkin(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                  const int32_t* agg, int64_t nc, int64_t* rp_c, int32_t* col_c, double* val_c) {
  Csr A = csr_copy(n, rp, ci, v);
  std::vector<int32_t> ag(agg, agg + n), mem;
  std::vector<int> cnt(nc, 0);
  int stride = 1;
  for (int64_t i = 0; i < n; ++i) stride = std::max(stride, ++cnt[ag[i]]);
  members_of(ag, nc, stride, mem);
  Csr Ac;
  galerkin(A, ag, nc, mem, stride, Ac);
  std::memcpy(rp_c, Ac.rowptr.data(), sizeof(int64_t) * (nc + 1));
  if (col_c) std::memcpy(col_c, Ac.col.data(), sizeof(int32_t) * Ac.col.size());
  if (val_c) std::memcpy(val_c, Ac.val.data(), sizeof(double) * Ac.val.size());
}

int orc_cholesky(int64_t n, const double* a, double* L) {
  std::vector<double> A(a, a + n * n), Lv;
  int st = cholesky(n, A, Lv);
  std::memcpy(L, Lv.data(), sizeof(double) * n * n);
  return st;
}

void orc_chol_solve(int64_t n, const double* L, const double* b, double* x) {
  std::vector<double> Lv(L, L + n * n);
  chol_solve(n, Lv, b, x);
}

// ---- hierarchy handle
void* orc_setup(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, int sweeps,
                int64_t max_coarse, int max_levels, double stall, int64_t max_dense,
                const double* omega, int* status) {
  Hierarchy* H = new Hierarchy();
  *status = build(*H, csr_copy(n, rp, ci, v), sweeps, max_coarse, max_levels, stall, max_dense,
                  omega);
  return H;
}

// orc_setup with smoothed prolongators (smooth_p = 1, Sec. 2.3).
void* orc_setup_smoothed(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                         int sweeps, int64_t max_coarse, int max_levels, double stall,
                         int64_t max_dense, int* status) {
  Hierarchy* H = new Hierarchy();
  *status = build(*H, csr_copy(n, rp, ci, v), sweeps, max_coarse, max_levels, stall, max_dense,
                  nullptr, std::vector<int64_t>(), nullptr, 1);
  return H;
}

// orc_setup with every hierarchy option: smoothed prolongators (smooth_p,
// smoothed with A_F when pfilter > 0) and the aggregation (0 matching sweeps,
// 1 VBM with strength theta).
void* orc_setup_general(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                        int sweeps, int64_t max_coarse, int max_levels, double stall,
                        int64_t max_dense, int smooth_p, int aggregation, double theta,
                        double pfilter, int* status) {
  Hierarchy* H = new Hierarchy();
  *status = build(*H, csr_copy(n, rp, ci, v), sweeps, max_coarse, max_levels, stall, max_dense,
                  nullptr, std::vector<int64_t>(), nullptr, smooth_p, aggregation, theta,
                  pfilter);
  return H;
}

// VBM aggregates of one matrix; returns their count.
int64_t orc_vbm_aggregate(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                          double theta, int32_t* agg) {
  std::vector<int32_t> a;
  const int64_t nc = vbm_aggregate(csr_copy(n, rp, ci, v), theta, a);
  std::memcpy(agg, a.data(), sizeof(int32_t) * n);
  return nc;
}

// P (n x n_c, smoothed) of level l and its damping w; rp/ci/v null to get nnz.
int64_t orc_level_prolongator(void* h, int l, int64_t* rp, int32_t* ci, double* v, double* w) {
  const Level& L = ((Hierarchy*)h)->lev[l];
  if (w) *w = L.wp;
  if (rp) std::memcpy(rp, L.P.rowptr.data(), sizeof(int64_t) * (L.P.n + 1));
  if (ci) std::memcpy(ci, L.P.col.data(), sizeof(int32_t) * L.P.nnz());
  if (v) std::memcpy(v, L.P.val.data(), sizeof(double) * L.P.nnz());
  return L.P.nnz();
}

// Hierarchy of nsys systems stacked block diagonally (sys_off: nsys + 1 row
// offsets); coarsening stops when every system has <= max_coarse rows.
void* orc_setup_systems(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                        int nsys, const int64_t* sys_off, int sweeps, int64_t max_coarse,
                        int max_levels, double stall, int64_t max_dense, int* status) {
  Hierarchy* H = new Hierarchy();
  std::vector<int64_t> sys(sys_off, sys_off + nsys + 1);
  *status = build(*H, csr_copy(n, rp, ci, v), sweeps, max_coarse, max_levels, stall, max_dense,
                  nullptr, sys);
  return H;
}

// A hierarchy for new values of the matrix `like` was built from (same
// sparsity): like's aggregates on every level, new Galerkin values, smoother
// scales and coarse factor.  -1 if the structure differs.
void* orc_setup_reuse(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                      void* like, int64_t max_dense, int* status) {
  const Hierarchy* L = (const Hierarchy*)like;
  Hierarchy* H = new Hierarchy();
  Csr A = csr_copy(n, rp, ci, v);
  const Csr& A0 = L->lev[0].A;
  if (A.n != A0.n || A.rowptr != A0.rowptr || A.col != A0.col) {
    *status = -1;
    return H;
  }
  *status = build(*H, std::move(A), L->sweeps, 0, 0, 0.0, max_dense, nullptr,
                  std::vector<int64_t>(), L);
  H->nu0 = L->nu0;
  H->variable = L->variable;
  H->coarse = L->coarse;
  H->coarse_maxit = L->coarse_maxit;
  H->coarse_tol = L->coarse_tol;
  return H;
}

// Cycle parameters of a hierarchy (defaults: V(1,1), dense Cholesky coarsest).
void orc_set_cycle(void* h, int nu0, int variable, int coarse, int coarse_maxit,
                   double coarse_tol) {
  Hierarchy* H = (Hierarchy*)h;
  H->nu0 = nu0;
  H->variable = variable;
  H->coarse = coarse;
  H->coarse_maxit = coarse_maxit;
  H->coarse_tol = coarse_tol;
}

void orc_free(void* h) { delete (Hierarchy*)h; }

int orc_levels(void* h) { return (int)((Hierarchy*)h)->lev.size(); }

int64_t orc_level_n(void* h, int l) { return ((Hierarchy*)h)->lev[l].A.n; }

int64_t orc_level_nnz(void* h, int l) { return ((Hierarchy*)h)->lev[l].A.nnz(); }

void orc_level_csr(void* h, int l, int64_t* rp, int32_t* ci, double* v) {
  const Csr& A = ((Hierarchy*)h)->lev[l].A;
  std::memcpy(rp, A.rowptr.data(), sizeof(int64_t) * (A.n + 1));
  std::memcpy(ci, A.col.data(), sizeof(int32_t) * A.nnz());
  std::memcpy(v, A.val.data(), sizeof(double) * A.nnz());
}

void orc_level_agg(void* h, int l, int32_t* agg) {
  const Level& L = ((Hierarchy*)h)->lev[l];
  std::memcpy(agg, L.agg.data(), sizeof(int32_t) * L.agg.size());
}

void orc_level_dinv(void* h, int l, double* d) {
  const Level& L = ((Hierarchy*)h)->lev[l];
  std::memcpy(d, L.dinv.data(), sizeof(double) * L.dinv.size());
}

void orc_coarse_factor(void* h, double* L) {
  const Hierarchy* H = (Hierarchy*)h;
  std::memcpy(L, H->chol.data(), sizeof(double) * H->chol.size());
}

void orc_vcycle(void* h, const double* r, double* z) { vcycle(*(Hierarchy*)h, 0, r, z); }

// PCG preconditioned by the V-cycle (h != nullptr), by a dense matrix
// (binv != nullptr, row-major n x n), or unpreconditioned (both null).
// out = {iterations, status, relres, true_relres}.
void orc_pcg(void* h, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
             const double* binv, const double* b, double* x, double tol, int maxit,
             int beta_form, double* res_hist, double* x_hist, double* out) {
  Csr A = csr_copy(n, rp, ci, v);
  std::function<void(const double*, double*)> prec;
  if (h) {
    Hierarchy* H = (Hierarchy*)h;
    prec = [H](const double* r, double* z) { vcycle(*H, 0, r, z); };
  } else if (binv) {
    prec = [n, binv](const double* r, double* z) {
      for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = 0; k < n; ++k) s += binv[i * n + k] * r[k];
        z[i] = s;
      }
    };
  } else {
    prec = [n](const double* r, double* z) { std::memcpy(z, r, sizeof(double) * n); };
  }
  PcgOut o = pcg(A, prec, b, x, tol, maxit, beta_form, res_hist, x_hist);
  out[0] = o.iters;
  out[1] = o.status;
  out[2] = o.relres;
  out[3] = o.true_relres;
}

// PCG on the diagonal block rows/columns [r0, r1) of the hierarchy's level-0
// matrix (which must have no entry coupling the block to other rows),
// preconditioned by the hierarchy's V-cycle applied to the block's residual
// padded with zeros.  Returns -1 in out[1] if the block is coupled.
void orc_pcg_block(void* h, int64_t r0, int64_t r1, const double* b, double* x, double tol,
                   int maxit, int beta_form, double* out) {
  Hierarchy* H = (Hierarchy*)h;
  const Csr& A0 = H->lev[0].A;
  const int64_t N = A0.n, m = r1 - r0;
  Csr S;
  S.n = m;
  S.rowptr.assign(m + 1, 0);
  for (int64_t i = r0; i < r1; ++i) {
    for (int64_t e = A0.rowptr[i]; e < A0.rowptr[i + 1]; ++e) {
      const int64_t j = A0.col[e];
      if (j < r0 || j >= r1) {
        out[1] = -1;
        return;
      }
      S.col.push_back((int32_t)(j - r0));
      S.val.push_back(A0.val[e]);
    }
    S.rowptr[i - r0 + 1] = (int64_t)S.col.size();
  }
  auto prec = [H, r0, m, N](const double* r, double* z) {
    std::vector<double> full(N, 0.0), zf(N);
    std::memcpy(full.data() + r0, r, sizeof(double) * m);
    vcycle(*H, 0, full.data(), zf.data());
    std::memcpy(z, zf.data() + r0, sizeof(double) * m);
  };
  PcgOut o = pcg(S, prec, b, x, tol, maxit, beta_form, nullptr, nullptr);
  out[0] = o.iters;
  out[1] = o.status;
  out[2] = o.relres;
  out[3] = o.true_relres;
}

}  // extern "C"
