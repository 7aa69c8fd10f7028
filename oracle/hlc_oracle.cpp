// hlc_oracle.cpp -- TEST INFRASTRUCTURE ONLY.
//
// Plain, slow, FP64 CPU oracle for one evaluation of the Gaussian
// log-likelihood of a Matern random field with hierarchical (H-) matrices,
// written from arXiv:1709.08625 (HLIBCov).  It shares no code with the CUDA
// library: no headers, helpers, tables or generators.  Only the test suite,
// the smoke check and the benchmark's CPU-baseline leg may load it; the
// product path never does.
//
// What is here, and the passage each part follows:
//   * Matern covariance, eq. (3) (Sec. 2.1), with the nugget of eq. (4)
//     (Sec. 4.1) on the diagonal.
//   * Dense reference: eq. (1) evaluated with a hand-written blocked Cholesky
//     (log det C = 2 sum log L_ii, quadratic form through L w = z).
//   * H-matrix path (Sec. 2.2, Def. 2.2, App. A):
//       - cluster tree by recursive geometric bisection of Morton-sorted
//         points (Sec. 2.2: rows split into two sub-sets down to n_min),
//       - block-cluster tree with the standard admissibility condition
//         min(diam B_t, diam B_s) <= eta dist(B_t, B_s) (App. A),
//       - dense inadmissible leaves, admissible leaves by ACA (App. B) and
//         QR+SVD recompression (Remark A.1) to block accuracy eps (Sec. 2.2),
//       - recursive H-Cholesky built from the H-arithmetic of Table 1
//         (truncated add and multiply-add), eq. (2) for the likelihood,
//       - forward/backward H-solves, the H-matvec, and the conjugate
//         gradients on C~ preconditioned with the factor (App. B listing).
//
// Parity pins live in tests/test_oracle_pins.py (closed forms, Bessel
// identities and library values, brute-force determinants, invariants).
//
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -shared -fPIC.
// -ffp-contract=off keeps the geometry (Morton quantisation, admissibility)
// bit-identical across x86 and Arm hosts.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Matern covariance, eq. (3):
//   C(h) = sigma2 / (2^(nu-1) Gamma(nu)) * (h/ell)^nu * K_nu(h/ell)
// The limit h -> 0 is sigma2, since x^nu K_nu(x) -> 2^(nu-1) Gamma(nu).
// ---------------------------------------------------------------------------
struct Theta {
  double sigma2, ell, nu, nugget;
};

double matern_bessel(double h, const Theta& th) {
  if (h == 0.0) return th.sigma2;
  const double x = h / th.ell;
  // Below 1e-100 every correction term of the small-x expansion of
  // x^nu K_nu(x) is under 1e-60 relative for nu >= 0.3: the value is the limit.
  if (x < 1e-100) return th.sigma2;
  const double k = std::cyl_bessel_k(th.nu, x);
  if (k == 0.0) return 0.0;  // K_nu underflowed (x > ~700)
  return th.sigma2 / (std::pow(2.0, th.nu - 1.0) * std::tgamma(th.nu)) *
         std::pow(x, th.nu) * k;
}

// The same function with the half-integer closed forms of K_nu substituted:
//   nu = 1/2: K_{1/2}(x) = sqrt(pi/(2x)) e^-x, Gamma(1/2) = sqrt(pi)
//             => C = sigma2 e^-x
//   nu = 3/2: K_{3/2}(x) = sqrt(pi/(2x)) e^-x (1 + 1/x), Gamma(3/2) = sqrt(pi)/2
//             => C = sigma2 (1 + x) e^-x
// Other nu use the Bessel form above.
double matern(double h, const Theta& th) {
  const double x = h / th.ell;
  if (th.nu == 0.5) return th.sigma2 * std::exp(-x);
  if (th.nu == 1.5) return th.sigma2 * (1.0 + x) * std::exp(-x);
  return matern_bessel(h, th);
}

double pdist(double x0, double y0, double x1, double y1) {
  const double dx = x0 - x1, dy = y0 - y1;
  return std::sqrt(dx * dx + dy * dy);
}

// ---------------------------------------------------------------------------
// Small dense helpers (column-major).
// ---------------------------------------------------------------------------
struct Mat {
  long m = 0, n = 0;
  std::vector<double> a;
  Mat() = default;
  Mat(long m_, long n_) : m(m_), n(n_), a((size_t)m_ * (size_t)n_, 0.0) {}
  double& operator()(long i, long j) { return a[(size_t)i + (size_t)j * m]; }
  double operator()(long i, long j) const { return a[(size_t)i + (size_t)j * m]; }
  double* data() { return a.data(); }
};

// A view of a column-major block: element (i, j) at p[i + j * ld].
struct View {
  double* p;
  long m, n, ld;
  double& at(long i, long j) const { return p[i + j * ld]; }
  View rows(long r0, long r1) const { return View{p + r0, r1 - r0, n, ld}; }
};
View view(Mat& M) { return View{M.data(), M.m, M.n, M.m}; }

// Householder QR of A (m x K): thin Q (m x p), R (p x K), p = min(m, K).
void householder_qr(const Mat& A, Mat& Q, Mat& R) {
  const long m = A.m, K = A.n, p = std::min(m, K);
  Mat W = A;
  std::vector<std::vector<double>> vs;  // reflectors, vs[j] has length m - j
  vs.reserve(p);
  for (long j = 0; j < p; ++j) {
    double nrm2 = 0.0;
    for (long i = j; i < m; ++i) nrm2 += W(i, j) * W(i, j);
    const double nrm = std::sqrt(nrm2);
    std::vector<double> v(m - j, 0.0);
    if (nrm > 0.0) {
      const double alpha = (W(j, j) >= 0.0) ? -nrm : nrm;
      for (long i = j; i < m; ++i) v[i - j] = W(i, j);
      v[0] -= alpha;
      double vn2 = 0.0;
      for (double t : v) vn2 += t * t;
      if (vn2 > 0.0) {
        const double vn = std::sqrt(vn2);
        for (double& t : v) t /= vn;
        for (long c = j; c < K; ++c) {
          double d = 0.0;
          for (long i = j; i < m; ++i) d += v[i - j] * W(i, c);
          for (long i = j; i < m; ++i) W(i, c) -= 2.0 * v[i - j] * d;
        }
      } else {
        std::fill(v.begin(), v.end(), 0.0);
      }
    }
    vs.push_back(std::move(v));
  }
  R = Mat(p, K);
  for (long c = 0; c < K; ++c)
    for (long i = 0; i <= std::min(c, p - 1); ++i) R(i, c) = W(i, c);
  Q = Mat(m, p);
  for (long c = 0; c < p; ++c) Q(c, c) = 1.0;
  for (long j = p - 1; j >= 0; --j) {
    const std::vector<double>& v = vs[j];
    for (long c = 0; c < p; ++c) {
      double d = 0.0;
      for (long i = j; i < m; ++i) d += v[i - j] * Q(i, c);
      for (long i = j; i < m; ++i) Q(i, c) -= 2.0 * v[i - j] * d;
    }
  }
}

// One-sided (Hestenes) Jacobi SVD of B (p x q): B = X diag(S) Y^T with the
// singular values sorted in decreasing order; X is p x r, Y is q x r with
// r = min(p, q).  Rotations run on the narrower side (B or B^T).  A pair of
// columns is rotated while |gamma| > max(p, 16) 1e-14 sqrt(alpha beta): the
// columns end orthogonal to ~1e-13, far below any truncation threshold,
// without chasing the rounding noise of the length-p dot products; pairs of
// columns both below 1e-13 |B|_F are at rounding level, carry nothing above
// any truncation threshold and are left alone.
void jacobi_svd_cols(Mat& B, Mat& Y) {
  const long p = B.m, q = B.n;
  Y = Mat(q, q);
  for (long i = 0; i < q; ++i) Y(i, i) = 1.0;
  double fro2 = 0.0;
  for (double v : B.a) fro2 += v * v;
  const double tiny = 1e-26 * fro2;
  const double rtol = (double)std::max<long>(p, 16) * 1e-14;
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (long i = 0; i < q - 1; ++i) {
      for (long j = i + 1; j < q; ++j) {
        double a = 0.0, b = 0.0, g = 0.0;
        for (long k = 0; k < p; ++k) {
          a += B(k, i) * B(k, i);
          b += B(k, j) * B(k, j);
          g += B(k, i) * B(k, j);
        }
        if (a <= tiny && b <= tiny) continue;
        if (g == 0.0 || std::fabs(g) <= rtol * std::sqrt(a * b)) continue;
        rotated = true;
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) /
                         (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (long k = 0; k < p; ++k) {
          const double bi = B(k, i), bj = B(k, j);
          B(k, i) = c * bi - s * bj;
          B(k, j) = s * bi + c * bj;
        }
        for (long k = 0; k < q; ++k) {
          const double yi = Y(k, i), yj = Y(k, j);
          Y(k, i) = c * yi - s * yj;
          Y(k, j) = s * yi + c * yj;
        }
      }
    }
    if (!rotated) break;
  }
}

void jacobi_svd(const Mat& B0, Mat& X, std::vector<double>& S, Mat& Y) {
  const bool tr = B0.n > B0.m;  // orthogonalise the columns of the narrower side
  Mat B = tr ? Mat(B0.n, B0.m) : B0;
  if (tr)
    for (long j = 0; j < B0.n; ++j)
      for (long i = 0; i < B0.m; ++i) B(j, i) = B0(i, j);
  Mat J;
  jacobi_svd_cols(B, J);
  const long p = B.m, q = B.n;  // q <= p
  std::vector<double> sv(q);
  for (long j = 0; j < q; ++j) {
    double s2 = 0.0;
    for (long k = 0; k < p; ++k) s2 += B(k, j) * B(k, j);
    sv[j] = std::sqrt(s2);
  }
  std::vector<long> ord(q);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](long u, long v) { return sv[u] > sv[v]; });
  // B J = W diag(sv): left vectors W = B J / sv, right vectors J.
  Mat W(p, q), Js(q, q);
  S.assign(q, 0.0);
  for (long jj = 0; jj < q; ++jj) {
    const long j = ord[jj];
    S[jj] = sv[j];
    for (long k = 0; k < p; ++k) W(k, jj) = (sv[j] > 0.0) ? B(k, j) / sv[j] : 0.0;
    for (long k = 0; k < q; ++k) Js(k, jj) = J(k, j);
  }
  if (!tr) {  // B0 = W S Js^T
    X = W;
    Y = Js;
  } else {  // B0^T = W S Js^T  =>  B0 = Js S W^T
    X = Js;
    Y = W;
  }
}

// Truncation of R = U V^T (Remark A.1): QR of both factors, SVD of the
// small core R_u R_v^T, keep the singular values sigma_i > eps * sigma_1 --
// at most kfix of them in the fixed-rank mode of Tables 2 and 3 (kfix > 0).
// On return U is m x k, V is n x k with U V^T the truncated matrix.
void truncate_lr(Mat& U, Mat& V, double eps, long kfix = 0) {
  const long K = U.n;
  if (K == 0) return;
  Mat Qu, Ru, Qv, Rv;
  householder_qr(U, Qu, Ru);
  householder_qr(V, Qv, Rv);
  Mat M(Ru.m, Rv.m);  // Ru Rv^T
  for (long j = 0; j < Rv.m; ++j)
    for (long i = 0; i < Ru.m; ++i) {
      double s = 0.0;
      for (long c = 0; c < K; ++c) s += Ru(i, c) * Rv(j, c);
      M(i, j) = s;
    }
  Mat X, Y;
  std::vector<double> S;
  jacobi_svd(M, X, S, Y);
  long k = 0;
  if (!S.empty() && S[0] > 0.0)
    while (k < (long)S.size() && S[k] > eps * S[0]) ++k;
  if (kfix > 0 && k > kfix) k = kfix;
  Mat Un(U.m, k), Vn(V.m, k);
  for (long c = 0; c < k; ++c) {
    for (long i = 0; i < U.m; ++i) {
      double s = 0.0;
      for (long t = 0; t < Qu.n; ++t) s += Qu(i, t) * X(t, c);
      Un(i, c) = s * S[c];
    }
    for (long i = 0; i < V.m; ++i) {
      double s = 0.0;
      for (long t = 0; t < Qv.n; ++t) s += Qv(i, t) * Y(t, c);
      Vn(i, c) = s;
    }
  }
  U = std::move(Un);
  V = std::move(Vn);
}

// ---------------------------------------------------------------------------
// Dense blocked Cholesky (lower, column-major, in place).  Returns 0, or
// -(j+1) when pivot j is not positive (the NaN failure of Sec. 3).
// A pivot counts as non-positive when it is at rounding level: below
// 64 u times the diagonal entry it was reduced from (u = 2^-53).  Sec. 3
// traces the failure to diagonal entries "very close to zero"; with a nugget
// tau^2 > 0 every pivot is at least tau^2, far above this level.
// ---------------------------------------------------------------------------
constexpr double kPivotTol = 64.0 * 1.1102230246251565e-16;

long dense_cholesky(double* A, long n) {
  const long nb = 64;
  for (long k = 0; k < n; k += nb) {
    const long b = std::min(nb, n - k);
    // factor the diagonal block
    for (long j = k; j < k + b; ++j) {
      double d = A[j + j * n];
      const double d0 = d;
      for (long p = k; p < j; ++p) d -= A[j + p * n] * A[j + p * n];
      if (!(d > kPivotTol * d0)) return -(j + 1);
      d = std::sqrt(d);
      A[j + j * n] = d;
      for (long i = j + 1; i < k + b; ++i) {
        double s = A[i + j * n];
        for (long p = k; p < j; ++p) s -= A[i + p * n] * A[j + p * n];
        A[i + j * n] = s / d;
      }
    }
    // panel below: A21 := A21 L11^-T
#pragma omp parallel for schedule(static)
    for (long i = k + b; i < n; ++i) {
      for (long j = k; j < k + b; ++j) {
        double s = A[i + j * n];
        for (long p = k; p < j; ++p) s -= A[i + p * n] * A[j + p * n];
        A[i + j * n] = s / A[j + j * n];
      }
    }
    // trailing update of the lower triangle: A22 -= A21 A21^T
#pragma omp parallel for schedule(dynamic, 16)
    for (long j = k + b; j < n; ++j) {
      for (long p = k; p < k + b; ++p) {
        const double ljp = A[j + p * n];
        if (ljp == 0.0) continue;
        double* col = A + j * n;
        const double* lp = A + p * n;
        for (long i = j; i < n; ++i) col[i] -= lp[i] * ljp;
      }
    }
  }
  return 0;
}

void dense_cov(const double* x, const double* y, long n, const Theta& th, double* C) {
#pragma omp parallel for schedule(dynamic, 16)
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < n; ++i) {
      double v = matern(pdist(x[i], y[i], x[j], y[j]), th);
      if (i == j) v += th.nugget;
      C[i + j * n] = v;
    }
}

// ---------------------------------------------------------------------------
// Cluster tree and block-cluster tree (Sec. 2.2, App. A).
// ---------------------------------------------------------------------------
enum { DENSE = 0, LOWRANK = 1, SUBDIV = 2 };

struct Cluster {
  long lo, hi;
  double bmin[2], bmax[2];
  int child[2];
  int level;
  bool leaf() const { return child[0] < 0; }
  long size() const { return hi - lo; }
};

struct Block {
  int r = -1, s = -1;
  int type = DENSE;
  bool diag = false;
  // children: off-diagonal ch[2*i+j] = (r_i, s_j); diagonal ch[0] = (r0,r0),
  // ch[2] = (r1,r0), ch[3] = (r1,r1), ch[1] unused (upper part not stored).
  int ch[4] = {-1, -1, -1, -1};
  Mat D, U, V;
};

struct HTree {
  long n = 0;
  int leaf = 32;
  double eta = 2.0;
  std::vector<double> px, py;  // points in tree order
  std::vector<int> perm;       // tree position -> user index
  std::vector<Cluster> cl;
  std::vector<Block> C;  // assembled covariance (lower triangle)
  std::vector<Block> L;  // factor
  int depth = 0;
  Theta th{1, 1, 0.5, 0};
  double eps = 1e-6;
  long kfix = 0;  // fixed-rank mode (Tables 2 and 3): at most kfix columns per block
  int adm = 0;    // 0 standard (min diam), 1 max diam, 2 weak
  int split = 0;  // 0 geometric midpoint, 1 cardinality (median)
  bool assembled = false, factored = false;
};

// Morton key: quantise each coordinate over the global bounding box to 32
// bits, q = floor((c - min) / (max - min) * (2^32 - 1)), and interleave the
// bits with x in the even positions.
uint64_t morton_key(double cx, double cy, const double* lo, const double* hi) {
  uint32_t q[2];
  const double c[2] = {cx, cy};
  for (int d = 0; d < 2; ++d) {
    const double range = hi[d] - lo[d];
    if (range > 0.0) {
      const double t = (c[d] - lo[d]) / range * 4294967295.0;
      q[d] = (uint32_t)std::floor(t);
    } else {
      q[d] = 0u;
    }
  }
  uint64_t key = 0;
  for (int b = 0; b < 32; ++b) {
    key |= (uint64_t)((q[0] >> b) & 1u) << (2 * b);
    key |= (uint64_t)((q[1] >> b) & 1u) << (2 * b + 1);
  }
  return key;
}

// Recursive bisection: tight bounding box, its longest axis (x on ties).
// Geometric rule: coordinates <= the axis midpoint go left.  Cardinality rule
// (the "two equal sized sub-sets" of Sec. 2.2): the floor(size/2) points with
// the smallest coordinates go left, ties taken in the current order.  Both
// keep the current order within each side; stop at size <= leaf, or when a
// side would be empty.
int build_cluster(HTree& T, const double* x, const double* y, std::vector<int>& idx,
                  long lo, long hi, int level) {
  Cluster c;
  c.lo = lo;
  c.hi = hi;
  c.level = level;
  c.child[0] = c.child[1] = -1;
  c.bmin[0] = c.bmin[1] = INFINITY;
  c.bmax[0] = c.bmax[1] = -INFINITY;
  for (long i = lo; i < hi; ++i) {
    const double p[2] = {x[idx[i]], y[idx[i]]};
    for (int d = 0; d < 2; ++d) {
      c.bmin[d] = std::min(c.bmin[d], p[d]);
      c.bmax[d] = std::max(c.bmax[d], p[d]);
    }
  }
  const int id = (int)T.cl.size();
  T.cl.push_back(c);
  T.depth = std::max(T.depth, level);
  if (hi - lo <= T.leaf) return id;
  const double ex = c.bmax[0] - c.bmin[0], ey = c.bmax[1] - c.bmin[1];
  const int axis = (ex >= ey) ? 0 : 1;
  std::vector<int> left, right;
  if (T.split == 0) {
    const double mid = 0.5 * (c.bmin[axis] + c.bmax[axis]);
    for (long i = lo; i < hi; ++i) {
      const double v = axis == 0 ? x[idx[i]] : y[idx[i]];
      (v <= mid ? left : right).push_back(idx[i]);
    }
  } else {
    // positions of the cluster sorted by coordinate, ties by position
    std::vector<long> ord(hi - lo);
    std::iota(ord.begin(), ord.end(), lo);
    const double* co = axis == 0 ? x : y;
    std::stable_sort(ord.begin(), ord.end(), [&](long a, long b) { return co[idx[a]] < co[idx[b]]; });
    std::vector<char> goes_left(hi - lo, 0);
    for (long q = 0; q < (hi - lo) / 2; ++q) goes_left[ord[q] - lo] = 1;
    for (long i = lo; i < hi; ++i) (goes_left[i - lo] ? left : right).push_back(idx[i]);
  }
  if (left.empty() || right.empty()) return id;
  long pos = lo;
  for (int v : left) idx[pos++] = v;
  for (int v : right) idx[pos++] = v;
  const long cut = lo + (long)left.size();
  const int c0 = build_cluster(T, x, y, idx, lo, cut, level + 1);
  const int c1 = build_cluster(T, x, y, idx, cut, hi, level + 1);
  T.cl[id].child[0] = c0;
  T.cl[id].child[1] = c1;
  return id;
}

double box_diam(const Cluster& c) {
  const double ex = c.bmax[0] - c.bmin[0], ey = c.bmax[1] - c.bmin[1];
  return std::sqrt(ex * ex + ey * ey);
}

double box_dist(const Cluster& a, const Cluster& b) {
  double d2 = 0.0;
  for (int d = 0; d < 2; ++d) {
    const double g = std::max(0.0, std::max(a.bmin[d] - b.bmax[d], b.bmin[d] - a.bmax[d]));
    d2 += g * g;
  }
  return std::sqrt(d2);
}

// Admissibility (App. A) of two distinct clusters: standard
// min(diam) <= eta dist, or max(diam) <= eta dist, both with dist > 0; weak
// admissibility takes every such pair.
bool admissible(const HTree& T, int r, int s) {
  if (T.adm == 2) return true;
  const double dist = box_dist(T.cl[r], T.cl[s]);
  if (!(dist > 0.0)) return false;
  const double dr = box_diam(T.cl[r]), ds = box_diam(T.cl[s]);
  return (T.adm == 1 ? std::max(dr, ds) : std::min(dr, ds)) <= T.eta * dist;
}

// Block-cluster tree over the lower triangle (row cluster at or after the
// column cluster in tree order).
int build_block(HTree& T, std::vector<Block>& B, int r, int s) {
  const int id = (int)B.size();
  B.emplace_back();
  B[id].r = r;
  B[id].s = s;
  B[id].diag = (r == s);
  const Cluster& cr = T.cl[r];
  const Cluster& cs = T.cl[s];
  if (r == s) {
    if (cr.leaf()) {
      B[id].type = DENSE;
    } else {
      B[id].type = SUBDIV;
      const int a = build_block(T, B, cr.child[0], cr.child[0]);
      const int b = build_block(T, B, cr.child[1], cr.child[0]);
      const int c = build_block(T, B, cr.child[1], cr.child[1]);
      B[id].ch[0] = a;
      B[id].ch[2] = b;
      B[id].ch[3] = c;
    }
  } else if (admissible(T, r, s)) {
    B[id].type = LOWRANK;
  } else if (cr.leaf() || cs.leaf()) {
    B[id].type = DENSE;
  } else {
    B[id].type = SUBDIV;
    int kids[4];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) kids[2 * i + j] = build_block(T, B, cr.child[i], cs.child[j]);
    for (int q = 0; q < 4; ++q) B[id].ch[q] = kids[q];
  }
  return id;
}

void leaf_list(const std::vector<Block>& B, int b, std::vector<int>& out) {
  if (B[b].type != SUBDIV) {
    out.push_back(b);
    return;
  }
  for (int q = 0; q < 4; ++q)
    if (B[b].ch[q] >= 0) leaf_list(B, B[b].ch[q], out);
}

// ---------------------------------------------------------------------------
// Assembly: dense leaves exactly; admissible leaves by ACA with partial
// pivoting (App. B) followed by the recompression of Remark A.1.
// ---------------------------------------------------------------------------
double entry(const HTree& T, long i, long j) {
  double v = matern(pdist(T.px[i], T.py[i], T.px[j], T.py[j]), T.th);
  if (i == j) v += T.th.nugget;
  return v;
}

// ACA with partial pivoting.  Returns U (m x k) = residual columns and
// V (n x k) = residual rows divided by the pivot, so that U V^T reproduces the
// crosses.  Stops when |u_k| |v_k| <= eps |S_k|_F (running Frobenius norm of
// the approximant); a vanishing pivot row moves on to the next unused row,
// at most three times in a row.
void aca(const HTree& T, long r0, long m, long c0, long n, double eps, long kmax, Mat& U, Mat& V) {
  std::vector<std::vector<double>> us, vs;
  std::vector<char> row_used(m, 0), col_used(n, 0);
  long next = 0;
  double s2 = 0.0;
  int zero_tries = 0;
  const long kcap = std::min(std::min(m, n), kmax);
  while ((long)us.size() < kcap) {
    const long i = next;
    row_used[i] = 1;
    std::vector<double> row(n);
    for (long j = 0; j < n; ++j) {
      double v = entry(T, r0 + i, c0 + j);
      for (size_t l = 0; l < us.size(); ++l) v -= us[l][i] * vs[l][j];
      row[j] = v;
    }
    long jp = -1;
    double best = -1.0;
    for (long j = 0; j < n; ++j)
      if (!col_used[j] && std::fabs(row[j]) > best) {
        best = std::fabs(row[j]);
        jp = j;
      }
    if (jp < 0) break;
    if (best == 0.0) {
      if (++zero_tries > 3) break;
      long nx = -1;
      for (long t = 0; t < m; ++t)
        if (!row_used[t]) {
          nx = t;
          break;
        }
      if (nx < 0) break;
      next = nx;
      continue;
    }
    zero_tries = 0;
    const double piv = row[jp];
    std::vector<double> v(n), u(m);
    for (long j = 0; j < n; ++j) v[j] = row[j] / piv;
    for (long t = 0; t < m; ++t) {
      double val = entry(T, r0 + t, c0 + jp);
      for (size_t l = 0; l < us.size(); ++l) val -= us[l][t] * vs[l][jp];
      u[t] = val;
    }
    col_used[jp] = 1;
    double uu = 0.0, vv = 0.0;
    for (double t : u) uu += t * t;
    for (double t : v) vv += t * t;
    double cross = 0.0;
    for (size_t l = 0; l < us.size(); ++l) {
      double a = 0.0, b = 0.0;
      for (long t = 0; t < m; ++t) a += us[l][t] * u[t];
      for (long t = 0; t < n; ++t) b += vs[l][t] * v[t];
      cross += a * b;
    }
    s2 += 2.0 * cross + uu * vv;
    us.push_back(u);
    vs.push_back(v);
    if (std::sqrt(uu) * std::sqrt(vv) <= eps * std::sqrt(std::max(s2, 0.0))) break;
    long nx = -1;
    double bu = -1.0;
    for (long t = 0; t < m; ++t)
      if (!row_used[t] && std::fabs(u[t]) > bu) {
        bu = std::fabs(u[t]);
        nx = t;
      }
    if (nx < 0) break;
    next = nx;
  }
  const long k = (long)us.size();
  U = Mat(m, k);
  V = Mat(n, k);
  for (long l = 0; l < k; ++l) {
    for (long t = 0; t < m; ++t) U(t, l) = us[l][t];
    for (long t = 0; t < n; ++t) V(t, l) = vs[l][t];
  }
}

// ---------------------------------------------------------------------------
// H-arithmetic (Table 1) for the recursive H-Cholesky of eq. (2).
// ---------------------------------------------------------------------------
// A low-rank term of a product, placed at (roff, coff) inside the target.
struct Term {
  Mat U, V;
  long roff, coff;
};

struct HCtx {
  HTree* T;
  std::vector<Block>* B;
  double eps;
  long err = 0;
  // accumulated updates of low-rank blocks (see add_lr / flush)
  std::vector<std::vector<Term>>* pending = nullptr;
  const Cluster& cl(int c) const { return T->cl[c]; }
  Block& b(int i) { return (*B)[i]; }
  long rows(int i) { return cl(b(i).r).size(); }
  long cols(int i) { return cl(b(i).s).size(); }
};

// Parallel tasks only pay off for large targets.
bool big(HCtx& H, int c) { return H.rows(c) * H.cols(c) >= 64L * 1024; }

// Y += alpha * A X ; A off-diagonal (any type), X |s| x c, Y |r| x c.
void flush(HCtx& H, int b);

void hmul(HCtx& H, int a, const View& X, const View& Y, double alpha) {
  flush(H, a);
  Block& A = H.b(a);
  const long c = X.n;
  if (A.type == DENSE) {
    for (long j = 0; j < c; ++j)
      for (long k = 0; k < A.D.n; ++k) {
        const double xk = alpha * X.at(k, j);
        if (xk == 0.0) continue;
        for (long i = 0; i < A.D.m; ++i) Y.at(i, j) += A.D(i, k) * xk;
      }
  } else if (A.type == LOWRANK) {
    const long k = A.U.n;
    Mat Tm(k, c);
    for (long j = 0; j < c; ++j)
      for (long l = 0; l < k; ++l) {
        double s = 0.0;
        for (long t = 0; t < A.V.m; ++t) s += A.V(t, l) * X.at(t, j);
        Tm(l, j) = s;
      }
    for (long j = 0; j < c; ++j)
      for (long l = 0; l < k; ++l) {
        const double tl = alpha * Tm(l, j);
        for (long i = 0; i < A.U.m; ++i) Y.at(i, j) += A.U(i, l) * tl;
      }
  } else {
    const long r0 = H.cl(A.r).lo, s0 = H.cl(A.s).lo;
    for (int q = 0; q < 4; ++q) {
      const int cb = A.ch[q];
      if (cb < 0) continue;
      const Cluster& cr = H.cl(H.b(cb).r);
      const Cluster& cs = H.cl(H.b(cb).s);
      hmul(H, cb, X.rows(cs.lo - s0, cs.hi - s0), Y.rows(cr.lo - r0, cr.hi - r0), alpha);
    }
  }
}

// Y += alpha * A^T X ; A off-diagonal, X |r| x c, Y |s| x c.
void hmul_t(HCtx& H, int a, const View& X, const View& Y, double alpha) {
  flush(H, a);
  Block& A = H.b(a);
  const long c = X.n;
  if (A.type == DENSE) {
    for (long j = 0; j < c; ++j)
      for (long k = 0; k < A.D.n; ++k) {
        double s = 0.0;
        for (long i = 0; i < A.D.m; ++i) s += A.D(i, k) * X.at(i, j);
        Y.at(k, j) += alpha * s;
      }
  } else if (A.type == LOWRANK) {
    const long k = A.U.n;
    Mat Tm(k, c);
    for (long j = 0; j < c; ++j)
      for (long l = 0; l < k; ++l) {
        double s = 0.0;
        for (long t = 0; t < A.U.m; ++t) s += A.U(t, l) * X.at(t, j);
        Tm(l, j) = s;
      }
    for (long j = 0; j < c; ++j)
      for (long l = 0; l < k; ++l) {
        const double tl = alpha * Tm(l, j);
        for (long i = 0; i < A.V.m; ++i) Y.at(i, j) += A.V(i, l) * tl;
      }
  } else {
    const long r0 = H.cl(A.r).lo, s0 = H.cl(A.s).lo;
    for (int q = 0; q < 4; ++q) {
      const int cb = A.ch[q];
      if (cb < 0) continue;
      const Cluster& cr = H.cl(H.b(cb).r);
      const Cluster& cs = H.cl(H.b(cb).s);
      hmul_t(H, cb, X.rows(cr.lo - r0, cr.hi - r0), Y.rows(cs.lo - s0, cs.hi - s0), alpha);
    }
  }
}

// X := L^-1 X for a factored diagonal block L (forward substitution).
void trsv(HCtx& H, int l, const View& X) {
  Block& Ld = H.b(l);
  if (Ld.type == DENSE) {
    const long n = Ld.D.m;
    for (long j = 0; j < X.n; ++j)
      for (long i = 0; i < n; ++i) {
        double s = X.at(i, j);
        for (long p = 0; p < i; ++p) s -= Ld.D(i, p) * X.at(p, j);
        X.at(i, j) = s / Ld.D(i, i);
      }
    return;
  }
  const Cluster& t = H.cl(Ld.r);
  const Cluster& t0 = H.cl(H.cl(Ld.r).child[0]);
  const long cut = t0.hi - t.lo;
  const View X0 = X.rows(0, cut), X1 = X.rows(cut, X.m);
  trsv(H, Ld.ch[0], X0);
  hmul(H, Ld.ch[2], X0, X1, -1.0);
  trsv(H, Ld.ch[3], X1);
}

// X := L^-T X (backward substitution).
void trsv_t(HCtx& H, int l, const View& X) {
  Block& Ld = H.b(l);
  if (Ld.type == DENSE) {
    const long n = Ld.D.m;
    for (long j = 0; j < X.n; ++j)
      for (long i = n - 1; i >= 0; --i) {
        double s = X.at(i, j);
        for (long p = i + 1; p < n; ++p) s -= Ld.D(p, i) * X.at(p, j);
        X.at(i, j) = s / Ld.D(i, i);
      }
    return;
  }
  const Cluster& t = H.cl(Ld.r);
  const Cluster& t0 = H.cl(H.cl(Ld.r).child[0]);
  const long cut = t0.hi - t.lo;
  const View X0 = X.rows(0, cut), X1 = X.rows(cut, X.m);
  trsv_t(H, Ld.ch[3], X1);
  hmul_t(H, Ld.ch[2], X1, X0, -1.0);
  trsv_t(H, Ld.ch[0], X0);
}

void add_lr(HCtx& H, int c, const View& U, const View& V);
void add_dense(HCtx& H, int c, const View& P);

void add_terms(HCtx& H, int c, std::vector<Term>& terms);

// Accumulated updates: terms added to a low-rank block during the
// factorisation wait in a list and are truncated together (add_terms, in
// batches) right before the block is next read or rewritten, and at the end.
void queue_terms(HCtx& H, int c, std::vector<Term>& terms) {
  if (!H.pending) {
    add_terms(H, c, terms);
    return;
  }
  std::vector<Term>& q = (*H.pending)[c];
#pragma omp critical(hlc_pending)
  for (Term& t : terms) q.push_back(std::move(t));
}

void flush(HCtx& H, int b) {
  if (!H.pending || H.b(b).type != LOWRANK) return;
  std::vector<Term>& q = (*H.pending)[b];
  if (q.empty()) return;
  std::vector<Term> terms;
  terms.swap(q);
  add_terms(H, b, terms);
}

// Truncated sum (U, V) := trunc(U V^T + sum_t U_t V_t^T) of an m x n low-rank
// matrix (the truncated addition of Table 1), term by term in order: terms
// are taken in batches of at most kTruncBatch new columns (and at most 64
// terms; a wider term forms a batch of its own), acc := trunc(acc + batch),
// so that every core SVD stays small.  An empty (U, V) starts from zero.
constexpr long kTruncBatch = 64;

void trunc_sum(Mat& CU, Mat& CV, long m, long n, const std::vector<Term>& terms, double eps, long kfix) {
  size_t t0 = 0;
  while (t0 < terms.size()) {
    size_t t1 = t0;
    long kb = 0;
    while (t1 < terms.size() && (kb == 0 || kb + terms[t1].U.n <= kTruncBatch) && t1 - t0 < 64)
      kb += terms[t1++].U.n;
    const long K = CU.n + kb;
    Mat U(m, K), V(n, K);
    long col = 0;
    for (long l = 0; l < CU.n; ++l, ++col) {
      for (long i = 0; i < m; ++i) U(i, col) = CU(i, l);
      for (long i = 0; i < n; ++i) V(i, col) = CV(i, l);
    }
    for (size_t q = t0; q < t1; ++q) {
      const Term& t = terms[q];
      for (long l = 0; l < t.U.n; ++l, ++col) {
        for (long i = 0; i < t.U.m; ++i) U(t.roff + i, col) = t.U(i, l);
        for (long i = 0; i < t.V.m; ++i) V(t.coff + i, col) = t.V(i, l);
      }
    }
    truncate_lr(U, V, eps, kfix);
    CU = std::move(U);
    CV = std::move(V);
    t0 = t1;
  }
}

// Truncated sum of many terms into a low-rank block C (Table 1's truncated
// addition, applied to a sum whose order the paper leaves open).  Up to
// kTreeMinTerms - 1 terms are added in order (trunc_sum).  With more, the
// sum is formed as a balanced tree: the terms are split in order into
// groups of kTreeLeafTerms, each group is truncated on its own (S_g :=
// trunc(sum of the group)), adjacent partial sums are combined pairwise
// (S := trunc(S_a + S_b); an odd last one moves up unchanged) until two
// remain, and C := trunc(C + S_1 + S_2).  Every node truncates at eps; the
// grouping depends on the number of terms only.
constexpr size_t kTreeMinTerms = 9;
constexpr size_t kTreeLeafTerms = 4;

void add_terms(HCtx& H, int c, std::vector<Term>& terms) {
  Block& C = H.b(c);
  const long m = H.rows(c), n = H.cols(c);
  if (terms.size() < kTreeMinTerms) {
    trunc_sum(C.U, C.V, m, n, terms, H.eps, H.T->kfix);
    return;
  }
  std::vector<Term> level;
  for (size_t g = 0; g < terms.size(); g += kTreeLeafTerms) {
    const size_t e = std::min(terms.size(), g + kTreeLeafTerms);
    std::vector<Term> grp(terms.begin() + g, terms.begin() + e);
    Term s;
    s.U = Mat(m, 0);
    s.V = Mat(n, 0);
    s.roff = s.coff = 0;
    trunc_sum(s.U, s.V, m, n, grp, H.eps, H.T->kfix);
    level.push_back(std::move(s));
  }
  while (level.size() > 2) {
    std::vector<Term> next;
    for (size_t i = 0; i < level.size(); i += 2) {
      if (i + 1 == level.size()) {
        next.push_back(std::move(level[i]));
        break;
      }
      std::vector<Term> pair;
      pair.push_back(std::move(level[i]));
      pair.push_back(std::move(level[i + 1]));
      Term s;
      s.U = Mat(m, 0);
      s.V = Mat(n, 0);
      s.roff = s.coff = 0;
      trunc_sum(s.U, s.V, m, n, pair, H.eps, H.T->kfix);
      next.push_back(std::move(s));
    }
    level.swap(next);
  }
  trunc_sum(C.U, C.V, m, n, level, H.eps, H.T->kfix);
}

// C += U V^T (with truncation when C is low-rank).
void add_lr(HCtx& H, int c, const View& U, const View& V) {
  Block& C = H.b(c);
  if (U.n == 0) return;
  if (C.type == DENSE) {
    for (long j = 0; j < C.D.n; ++j)
      for (long l = 0; l < U.n; ++l) {
        const double v = V.at(j, l);
        for (long i = 0; i < C.D.m; ++i) C.D(i, j) += U.at(i, l) * v;
      }
  } else if (C.type == LOWRANK) {
    std::vector<Term> ts(1);
    ts[0].U = Mat(U.m, U.n);
    ts[0].V = Mat(V.m, V.n);
    for (long l = 0; l < U.n; ++l) {
      for (long i = 0; i < U.m; ++i) ts[0].U(i, l) = U.at(i, l);
      for (long i = 0; i < V.m; ++i) ts[0].V(i, l) = V.at(i, l);
    }
    ts[0].roff = ts[0].coff = 0;
    queue_terms(H, c, ts);
  } else {
    const long r0 = H.cl(C.r).lo, s0 = H.cl(C.s).lo;
    const bool spawn = big(H, c);
    for (int q = 0; q < 4; ++q) {
      const int cb = C.ch[q];
      if (cb < 0) continue;
      const Cluster& cr = H.cl(H.b(cb).r);
      const Cluster& cs = H.cl(H.b(cb).s);
      const View Us = U.rows(cr.lo - r0, cr.hi - r0), Vs = V.rows(cs.lo - s0, cs.hi - s0);
#pragma omp task default(shared) firstprivate(cb, Us, Vs) if (spawn)
      add_lr(H, cb, Us, Vs);
    }
#pragma omp taskwait
  }
}

// C += P for a dense |r| x |s| matrix P (only the stored lower part of a
// diagonal target receives it).
void add_dense(HCtx& H, int c, const View& P) {
  Block& C = H.b(c);
  if (C.type == DENSE) {
    for (long j = 0; j < C.D.n; ++j)
      for (long i = 0; i < C.D.m; ++i) C.D(i, j) += P.at(i, j);
  } else if (C.type == LOWRANK) {
    // P as a low-rank term of rank min(|r|, |s|): P = I * P^T^T or P * I^T.
    std::vector<Term> ts(1);
    Term& t = ts[0];
    t.roff = t.coff = 0;
    if (P.m <= P.n) {
      t.U = Mat(P.m, P.m);
      t.V = Mat(P.n, P.m);
      for (long i = 0; i < P.m; ++i) t.U(i, i) = 1.0;
      for (long i = 0; i < P.m; ++i)
        for (long j = 0; j < P.n; ++j) t.V(j, i) = P.at(i, j);
    } else {
      t.U = Mat(P.m, P.n);
      t.V = Mat(P.n, P.n);
      for (long j = 0; j < P.n; ++j) t.V(j, j) = 1.0;
      for (long j = 0; j < P.n; ++j)
        for (long i = 0; i < P.m; ++i) t.U(i, j) = P.at(i, j);
    }
    queue_terms(H, c, ts);
  } else {
    const long r0 = H.cl(C.r).lo, s0 = H.cl(C.s).lo;
    for (int q = 0; q < 4; ++q) {
      const int cb = C.ch[q];
      if (cb < 0) continue;
      const Cluster& cr = H.cl(H.b(cb).r);
      const Cluster& cs = H.cl(H.b(cb).s);
      View sub{P.p + (cr.lo - r0) + (cs.lo - s0) * P.ld, cr.size(), cs.size(), P.ld};
      add_dense(H, cb, sub);
    }
  }
}

// Dense transpose copy of a dense block.
Mat transpose(const Mat& A) {
  Mat T(A.n, A.m);
  for (long j = 0; j < A.n; ++j)
    for (long i = 0; i < A.m; ++i) T(j, i) = A(i, j);
  return T;
}

// The exact product A B^T (A = (r, s), B = (r', s)) as a list of low-rank
// terms placed inside the |r| x |r'| target.
void prod_terms(HCtx& H, int a, int bb, long roff, long coff, std::vector<Term>& out) {
  flush(H, a);
  flush(H, bb);
  Block& A = H.b(a);
  Block& B = H.b(bb);
  const long ra = H.rows(a), rb = H.rows(bb);
  if (A.type == LOWRANK) {
    Term t;
    t.roff = roff;
    t.coff = coff;
    t.U = A.U;
    t.V = Mat(rb, A.V.n);
    Mat Vc = A.V;
    hmul(H, bb, view(Vc), view(t.V), 1.0);
    out.push_back(std::move(t));
  } else if (B.type == LOWRANK) {
    Term t;
    t.roff = roff;
    t.coff = coff;
    t.V = B.U;
    t.U = Mat(ra, B.V.n);
    Mat Vc = B.V;
    hmul(H, a, view(Vc), view(t.U), 1.0);
    out.push_back(std::move(t));
  } else if (A.type == DENSE && B.type == DENSE) {
    Term t;
    t.roff = roff;
    t.coff = coff;
    t.U = A.D;
    t.V = B.D;
    out.push_back(std::move(t));
  } else if (A.type == DENSE) {
    Term t;
    t.roff = roff;
    t.coff = coff;
    t.U = Mat(ra, ra);
    for (long i = 0; i < ra; ++i) t.U(i, i) = 1.0;
    Mat At = transpose(A.D);
    t.V = Mat(rb, ra);
    hmul(H, bb, view(At), view(t.V), 1.0);
    out.push_back(std::move(t));
  } else if (B.type == DENSE) {
    Term t;
    t.roff = roff;
    t.coff = coff;
    t.V = Mat(rb, rb);
    for (long i = 0; i < rb; ++i) t.V(i, i) = 1.0;
    Mat Bt = transpose(B.D);
    t.U = Mat(ra, rb);
    hmul(H, a, view(Bt), view(t.U), 1.0);
    out.push_back(std::move(t));
  } else {
    const long ar0 = H.cl(A.r).lo, br0 = H.cl(B.r).lo;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j)
        for (int l = 0; l < 2; ++l) {
          const int ai = H.b(a).ch[2 * i + l], bj = H.b(bb).ch[2 * j + l];
          prod_terms(H, ai, bj, roff + H.cl(H.b(ai).r).lo - ar0, coff + H.cl(H.b(bj).r).lo - br0, out);
        }
  }
}

// C += alpha * A B^T with truncation; A = (r, s), B = (r', s), C = (r, r').
void mul_add(HCtx& H, int c, int a, int bb, double alpha) {
  flush(H, a);
  flush(H, bb);
  const int ta = H.b(a).type, tb = H.b(bb).type, tc = H.b(c).type;
  const long ra = H.rows(a), rb = H.rows(bb);
  if (ta == LOWRANK) {
    Mat W(rb, H.b(a).V.n);
    Mat Vc = H.b(a).V;
    hmul(H, bb, view(Vc), view(W), 1.0);
    Mat U = H.b(a).U;
    for (double& v : U.a) v *= alpha;
    add_lr(H, c, view(U), view(W));
  } else if (tb == LOWRANK) {
    Mat W(ra, H.b(bb).V.n);
    Mat Vc = H.b(bb).V;
    hmul(H, a, view(Vc), view(W), alpha);
    Mat U = H.b(bb).U;
    add_lr(H, c, view(W), view(U));
  } else if (ta == DENSE && tb == DENSE) {
    const Mat& Ad = H.b(a).D;
    const Mat& Bd = H.b(bb).D;
    Mat P(ra, rb);
    for (long j = 0; j < rb; ++j)
      for (long k = 0; k < Ad.n; ++k) {
        const double v = alpha * Bd(j, k);
        for (long i = 0; i < ra; ++i) P(i, j) += Ad(i, k) * v;
      }
    add_dense(H, c, view(P));
  } else if (ta == DENSE) {
    Mat At = transpose(H.b(a).D);
    Mat W(rb, ra);
    hmul(H, bb, view(At), view(W), alpha);
    Mat P = transpose(W);
    add_dense(H, c, view(P));
  } else if (tb == DENSE) {
    Mat Bt = transpose(H.b(bb).D);
    Mat W(ra, rb);
    hmul(H, a, view(Bt), view(W), alpha);
    add_dense(H, c, view(W));
  } else if (tc == SUBDIV) {
    // The child targets are disjoint: update them as independent tasks; the
    // two contributions to one child stay in order.
    const bool dg = H.b(c).diag;
    const bool spawn = big(H, c);
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        if (dg && j > i) continue;
        const int cc = H.b(c).ch[2 * i + j];
        const int a0 = H.b(a).ch[2 * i], a1 = H.b(a).ch[2 * i + 1];
        const int b0 = H.b(bb).ch[2 * j], b1 = H.b(bb).ch[2 * j + 1];
#pragma omp task default(shared) firstprivate(cc, a0, a1, b0, b1) if (spawn)
        {
          mul_add(H, cc, a0, b0, alpha);
          mul_add(H, cc, a1, b1, alpha);
        }
      }
#pragma omp taskwait
  } else {
    std::vector<Term> terms;
    prod_terms(H, a, bb, 0, 0, terms);
    if (alpha != 1.0)
      for (Term& t : terms)
        for (double& v : t.U.a) v *= alpha;
    if (tc == LOWRANK) {
      queue_terms(H, c, terms);
    } else {
      Mat P(ra, rb);
      for (const Term& t : terms)
        for (long j = 0; j < t.V.m; ++j)
          for (long l = 0; l < t.U.n; ++l) {
            const double v = t.V(j, l);
            for (long i = 0; i < t.U.m; ++i) P(t.roff + i, t.coff + j) += t.U(i, l) * v;
          }
      add_dense(H, c, view(P));
    }
  }
}

// B := B L^-T for an off-diagonal block B = (r, s) and factored L = (s, s).
void trsm(HCtx& H, int l, int bb) {
  flush(H, bb);
  Block& B = H.b(bb);
  if (B.type == DENSE) {
    Mat Xt = transpose(B.D);
    trsv(H, l, view(Xt));
    H.b(bb).D = transpose(Xt);
  } else if (B.type == LOWRANK) {
    trsv(H, l, view(H.b(bb).V));
  } else {
    const Block& Ld = H.b(l);
    const int l00 = Ld.ch[0], l10 = Ld.ch[2], l11 = Ld.ch[3];
    const bool spawn = big(H, bb);
    for (int i = 0; i < 2; ++i) {  // the two block rows are independent
      const int b0 = H.b(bb).ch[2 * i + 0], b1 = H.b(bb).ch[2 * i + 1];
#pragma omp task default(shared) firstprivate(b0, b1) if (spawn)
      {
        trsm(H, l00, b0);
        mul_add(H, b1, b0, l10, -1.0);
        trsm(H, l11, b1);
      }
    }
#pragma omp taskwait
  }
}

// Recursive H-Cholesky of a diagonal block (in place).
void chol(HCtx& H, int m) {
  if (H.err) return;
  Block& M = H.b(m);
  if (M.type == DENSE) {
    const long n = M.D.m;
    for (long j = 0; j < n; ++j) {
      double d = M.D(j, j);
      const double d0 = d;
      for (long p = 0; p < j; ++p) d -= M.D(j, p) * M.D(j, p);
      if (!(d > kPivotTol * d0)) {
        H.err = -(H.cl(M.r).lo + j + 1);
        return;
      }
      d = std::sqrt(d);
      M.D(j, j) = d;
      for (long i = j + 1; i < n; ++i) {
        double s = M.D(i, j);
        for (long p = 0; p < j; ++p) s -= M.D(i, p) * M.D(j, p);
        M.D(i, j) = s / d;
      }
    }
    return;
  }
  const int m00 = M.ch[0], m10 = M.ch[2], m11 = M.ch[3];
  chol(H, m00);
  if (H.err) return;
  trsm(H, m00, m10);
  mul_add(H, m11, m10, m10, -1.0);
  chol(H, m11);
}

// y += C x for the symmetric matrix stored as its lower block triangle.
void symv(HCtx& H, int b, const View& x, const View& y) {
  Block& B = H.b(b);
  const Cluster& cr = H.cl(B.r);
  const Cluster& cs = H.cl(B.s);
  if (B.diag) {
    if (B.type == DENSE) {
      for (long j = 0; j < B.D.n; ++j) {
        const double xj = x.at(cs.lo + j, 0);
        for (long i = 0; i < B.D.m; ++i) y.at(cr.lo + i, 0) += B.D(i, j) * xj;
      }
    } else {
      symv(H, B.ch[0], x, y);
      symv(H, B.ch[2], x, y);
      symv(H, B.ch[3], x, y);
    }
    return;
  }
  hmul(H, b, x.rows(cs.lo, cs.hi), y.rows(cr.lo, cr.hi), 1.0);
  hmul_t(H, b, x.rows(cr.lo, cr.hi), y.rows(cs.lo, cs.hi), 1.0);
}

void stats(const HTree& T, const std::vector<Block>& B, long* max_rank, long* entries) {
  std::vector<int> lv;
  leaf_list(B, 0, lv);
  *max_rank = 0;
  *entries = 0;
  for (int b : lv) {
    if (B[b].type == DENSE) {
      *entries += B[b].D.m * B[b].D.n;
    } else {
      *max_rank = std::max(*max_rank, B[b].U.n);
      *entries += (B[b].U.m + B[b].V.m) * B[b].U.n;
    }
  }
  (void)T;
}

}  // namespace

// ===========================================================================
// C interface (ctypes).  Status: 0 ok, -1 bad argument, -2 not positive
// definite, -3 not assembled / not factored.
// ===========================================================================
extern "C" {

int orc_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Matern values at distances h[cnt]; use_bessel = 1 forces the K_nu form.
int orc_matern(const double* h, long cnt, double sigma2, double ell, double nu, int use_bessel,
               double* out) {
  if (!(ell > 0.0) || !(nu > 0.0) || cnt < 0) return -1;
  const Theta th{sigma2, ell, nu, 0.0};
  for (long i = 0; i < cnt; ++i) out[i] = use_bessel ? matern_bessel(h[i], th) : matern(h[i], th);
  return 0;
}

// Dense covariance (full n x n, column-major, nugget on the diagonal).
int orc_dense_cov(const double* x, const double* y, long n, double sigma2, double ell, double nu,
                  double nugget, double* C) {
  if (n < 0 || !(ell > 0.0) || !(nu > 0.0)) return -1;
  dense_cov(x, y, n, Theta{sigma2, ell, nu, nugget}, C);
  return 0;
}

// In-place blocked Cholesky of a full column-major n x n matrix (lower).
long orc_dense_cholesky(double* A, long n) { return dense_cholesky(A, n); }

// Dense eq. (1): out = {loglik, logdet, quad}.
long orc_dense_loglik(const double* x, const double* y, const double* z, long n, double sigma2,
                      double ell, double nu, double nugget, double* out) {
  if (n <= 0 || !(ell > 0.0) || !(nu > 0.0)) return -1;
  std::vector<double> A((size_t)n * n);
  dense_cov(x, y, n, Theta{sigma2, ell, nu, nugget}, A.data());
  const long st = dense_cholesky(A.data(), n);
  if (st != 0) return -2;
  double logdet = 0.0;
  for (long i = 0; i < n; ++i) logdet += 2.0 * std::log(A[i + i * n]);
  std::vector<double> w(z, z + n);
  for (long j = 0; j < n; ++j) {
    w[j] /= A[j + j * n];
    const double wj = w[j];
    for (long i = j + 1; i < n; ++i) w[i] -= A[i + j * n] * wj;
  }
  double quad = 0.0;
  for (long i = 0; i < n; ++i) quad += w[i] * w[i];
  out[0] = -0.5 * n * std::log(2.0 * M_PI) - 0.5 * logdet - 0.5 * quad;
  out[1] = logdet;
  out[2] = quad;
  return 0;
}

// z = L xi with C = L L^T the dense Cholesky factor (synthetic data of the
// kind the paper draws in Sec. 5.1).
long orc_dense_chol_apply(const double* x, const double* y, const double* xi, long n, double sigma2,
                          double ell, double nu, double nugget, double* z) {
  if (n <= 0) return -1;
  std::vector<double> A((size_t)n * n);
  dense_cov(x, y, n, Theta{sigma2, ell, nu, nugget}, A.data());
  if (dense_cholesky(A.data(), n) != 0) return -2;
  for (long i = 0; i < n; ++i) {
    double s = 0.0;
    for (long j = 0; j <= i; ++j) s += A[i + j * n] * xi[j];
    z[i] = s;
  }
  return 0;
}

void* orc_h_create(const double* x, const double* y, long n, int leaf, double eta, int adm, int split) {
  if (n <= 0 || leaf < 1 || !(eta > 0.0) || adm < 0 || adm > 2 || split < 0 || split > 1) return nullptr;
  HTree* T = new HTree();
  T->n = n;
  T->leaf = leaf;
  T->eta = eta;
  T->adm = adm;
  T->split = split;
  // Morton order over the global bounding box; ties by user index.
  double lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
  for (long i = 0; i < n; ++i) {
    lo[0] = std::min(lo[0], x[i]);
    hi[0] = std::max(hi[0], x[i]);
    lo[1] = std::min(lo[1], y[i]);
    hi[1] = std::max(hi[1], y[i]);
  }
  std::vector<uint64_t> key(n);
  for (long i = 0; i < n; ++i) key[i] = morton_key(x[i], y[i], lo, hi);
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return key[a] < key[b]; });
  build_cluster(*T, x, y, idx, 0, n, 0);
  T->perm = idx;
  T->px.resize(n);
  T->py.resize(n);
  for (long i = 0; i < n; ++i) {
    T->px[i] = x[idx[i]];
    T->py[i] = y[idx[i]];
  }
  build_block(*T, T->C, 0, 0);
  return T;
}

void orc_h_free(void* h) { delete static_cast<HTree*>(h); }

// info = {n, clusters, leaf clusters, dense leaves, low-rank leaves, depth}
int orc_h_info(void* h, long* info) {
  HTree* T = static_cast<HTree*>(h);
  long leaves = 0;
  for (const Cluster& c : T->cl) leaves += c.leaf() ? 1 : 0;
  std::vector<int> lv;
  leaf_list(T->C, 0, lv);
  long nd = 0, nl = 0;
  for (int b : lv) (T->C[b].type == DENSE ? nd : nl)++;
  info[0] = T->n;
  info[1] = (long)T->cl.size();
  info[2] = leaves;
  info[3] = nd;
  info[4] = nl;
  info[5] = T->depth;
  return 0;
}

int orc_h_perm(void* h, int* perm) {
  HTree* T = static_cast<HTree*>(h);
  std::copy(T->perm.begin(), T->perm.end(), perm);
  return 0;
}

// Clusters: lohi[2*i..] = {lo, hi}, bbox[4*i..] = {xmin, ymin, xmax, ymax},
// level[i], leaf flag in lohi sign (child count given separately).
long orc_h_clusters(void* h, long* lohi, double* bbox, int* level, int* is_leaf) {
  HTree* T = static_cast<HTree*>(h);
  for (size_t i = 0; i < T->cl.size(); ++i) {
    const Cluster& c = T->cl[i];
    lohi[2 * i] = c.lo;
    lohi[2 * i + 1] = c.hi;
    bbox[4 * i + 0] = c.bmin[0];
    bbox[4 * i + 1] = c.bmin[1];
    bbox[4 * i + 2] = c.bmax[0];
    bbox[4 * i + 3] = c.bmax[1];
    level[i] = c.level;
    is_leaf[i] = c.leaf() ? 1 : 0;
  }
  return (long)T->cl.size();
}

// Leaf blocks of the block-cluster tree: 5 longs each
// {row lo, row hi, col lo, col hi, type}; type 0 dense, 1 low-rank.
long orc_h_leaf_blocks(void* h, long* out) {
  HTree* T = static_cast<HTree*>(h);
  std::vector<int> lv;
  leaf_list(T->C, 0, lv);
  for (size_t q = 0; q < lv.size(); ++q) {
    const Block& b = T->C[lv[q]];
    out[5 * q + 0] = T->cl[b.r].lo;
    out[5 * q + 1] = T->cl[b.r].hi;
    out[5 * q + 2] = T->cl[b.s].lo;
    out[5 * q + 3] = T->cl[b.s].hi;
    out[5 * q + 4] = b.type;
  }
  return (long)lv.size();
}

// Assemble the H-matrix approximation of C (lower triangle).
int orc_h_assemble(void* h, double sigma2, double ell, double nu, double nugget, double eps,
                   long kmax) {
  HTree* T = static_cast<HTree*>(h);
  if (!(ell > 0.0) || !(nu > 0.0) || !(eps > 0.0)) return -1;
  T->th = Theta{sigma2, ell, nu, nugget};
  T->eps = eps;
  std::vector<int> lv;
  leaf_list(T->C, 0, lv);
#pragma omp parallel for schedule(dynamic, 1)
  for (long q = 0; q < (long)lv.size(); ++q) {
    Block& b = T->C[lv[q]];
    const Cluster& cr = T->cl[b.r];
    const Cluster& cs = T->cl[b.s];
    if (b.type == DENSE) {
      b.D = Mat(cr.size(), cs.size());
      for (long j = 0; j < cs.size(); ++j)
        for (long i = 0; i < cr.size(); ++i) b.D(i, j) = entry(*T, cr.lo + i, cs.lo + j);
      b.U = Mat();
      b.V = Mat();
    } else {
      // fixed-rank mode: ACA stops after kfix crosses
      const long kaca = T->kfix > 0 ? std::min<long>(kmax, T->kfix) : kmax;
      aca(*T, cr.lo, cr.size(), cs.lo, cs.size(), eps, kaca, b.U, b.V);
      truncate_lr(b.U, b.V, eps, T->kfix);
    }
  }
  T->assembled = true;
  T->factored = false;
  return 0;
}

// H-Cholesky of the assembled matrix (copy, then factor in place).
// accumulate = 1: updates of a low-rank block wait and are truncated together
// right before the block is next used; 0: every update is truncated at once.
long orc_h_cholesky(void* h, double eps, int accumulate) {
  HTree* T = static_cast<HTree*>(h);
  if (!T->assembled) return -3;
  T->L = T->C;
  std::vector<std::vector<Term>> pending(T->L.size());
  HCtx H{T, &T->L, eps};
  H.pending = accumulate ? &pending : nullptr;
#pragma omp parallel
#pragma omp single
  chol(H, 0);
  for (size_t b = 0; b < T->L.size(); ++b) flush(H, (int)b);
  if (H.err) {
    T->factored = false;
    return -2;
  }
  T->factored = true;
  return 0;
}

// stats = {max rank C, entries C, max rank L, entries L}
int orc_h_stats(void* h, long* st) {
  HTree* T = static_cast<HTree*>(h);
  st[0] = st[1] = st[2] = st[3] = 0;
  if (T->assembled) stats(*T, T->C, &st[0], &st[1]);
  if (T->factored) stats(*T, T->L, &st[2], &st[3]);
  return 0;
}

// Ranks of the low-rank leaves in leaf-list order (-1 for dense leaves).
long orc_h_ranks(void* h, int which, int* out) {
  HTree* T = static_cast<HTree*>(h);
  const std::vector<Block>& B = which ? T->L : T->C;
  std::vector<int> lv;
  leaf_list(T->C, 0, lv);
  for (size_t q = 0; q < lv.size(); ++q) out[q] = B[lv[q]].type == DENSE ? -1 : (int)B[lv[q]].U.n;
  return (long)lv.size();
}

// y = C~ x (which = 0) in user order.
int orc_h_matvec(void* h, const double* x, double* y) {
  HTree* T = static_cast<HTree*>(h);
  if (!T->assembled) return -3;
  const long n = T->n;
  std::vector<double> xt(n), yt(n, 0.0);
  for (long i = 0; i < n; ++i) xt[i] = x[T->perm[i]];
  HCtx H{T, &T->C, T->eps};
  symv(H, 0, View{xt.data(), n, 1, n}, View{yt.data(), n, 1, n});
  for (long i = 0; i < n; ++i) y[T->perm[i]] = yt[i];
  return 0;
}

// y = L~ x (trans = 0) or y = L~^T x (trans = 1) with the H-Cholesky factor
// L~ (the lower triangle of the factored block structure), in user order:
// the plain definition y_i = sum_j L~_ij x_j, taken leaf block by leaf
// block; a diagonal leaf contributes its lower triangle only.  Used to draw
// synthetic data Z = L~ xi (Sec. 5.1).
int orc_h_lmatvec(void* h, int trans, const double* x, double* y) {
  HTree* T = static_cast<HTree*>(h);
  if (!T->factored) return -3;
  const long n = T->n;
  std::vector<double> xt(n), yt(n, 0.0);
  for (long i = 0; i < n; ++i) xt[i] = x[T->perm[i]];
  std::vector<int> lv;
  leaf_list(T->L, 0, lv);
  for (int b : lv) {
    const Block& bl = T->L[b];
    const Cluster& cr = T->cl[bl.r];
    const Cluster& cs = T->cl[bl.s];
    const long m = cr.size(), nc = cs.size();
    // rows of the block map to cr, columns to cs; transposed, the other way
    const long in0 = trans ? cr.lo : cs.lo, out0 = trans ? cs.lo : cr.lo;
    if (bl.type == DENSE) {
      for (long j = 0; j < nc; ++j)
        for (long i = 0; i < m; ++i) {
          if (bl.diag && j > i) continue;
          if (!trans)
            yt[out0 + i] += bl.D(i, j) * xt[in0 + j];
          else
            yt[out0 + j] += bl.D(i, j) * xt[in0 + i];
        }
    } else {
      const long k = bl.U.n;
      for (long l = 0; l < k; ++l) {
        double w = 0.0;
        if (!trans) {
          for (long j = 0; j < nc; ++j) w += bl.V(j, l) * xt[in0 + j];
          for (long i = 0; i < m; ++i) yt[out0 + i] += bl.U(i, l) * w;
        } else {
          for (long i = 0; i < m; ++i) w += bl.U(i, l) * xt[in0 + i];
          for (long j = 0; j < nc; ++j) yt[out0 + j] += bl.V(j, l) * w;
        }
      }
    }
  }
  for (long i = 0; i < n; ++i) y[T->perm[i]] = yt[i];
  return 0;
}

// Expand C~ (which = 0) or L~ (which = 1) to a dense n x n column-major
// matrix in user order (small n only; C~ symmetric, L~ lower).
int orc_h_expand(void* h, int which, double* out) {
  HTree* T = static_cast<HTree*>(h);
  if (which == 0 && !T->assembled) return -3;
  if (which == 1 && !T->factored) return -3;
  const std::vector<Block>& B = which ? T->L : T->C;
  const long n = T->n;
  std::fill(out, out + n * n, 0.0);
  std::vector<int> lv;
  leaf_list(B, 0, lv);
  for (int b : lv) {
    const Block& bl = B[b];
    const Cluster& cr = T->cl[bl.r];
    const Cluster& cs = T->cl[bl.s];
    for (long j = 0; j < cs.size(); ++j)
      for (long i = 0; i < cr.size(); ++i) {
        double v;
        if (bl.type == DENSE) {
          v = bl.D(i, j);
        } else {
          v = 0.0;
          for (long l = 0; l < bl.U.n; ++l) v += bl.U(i, l) * bl.V(j, l);
        }
        const long gi = cr.lo + i, gj = cs.lo + j;
        if (which == 1 && bl.diag && j > i) v = 0.0;
        const long ui = T->perm[gi], uj = T->perm[gj];
        out[ui + uj * n] = v;
        if (which == 0 && gi != gj) out[uj + ui * n] = v;
      }
  }
  return 0;
}

// Likelihood from the factor, eq. (2), plus the quadratic form z^T C~^-1 z
// from conjugate gradients on C~ preconditioned with (L~ L~^T)^-1, the
// solver of the App. B listing (CG with the inverse factor as
// preconditioner), run to |z - C~ x| <= tol |z| or maxit iterations.
// out = {loglik, logdet, quad, quad_factor, iterations, rel_residual}
int orc_h_loglik(void* h, const double* z, double tol, int maxit, double* out) {
  HTree* T = static_cast<HTree*>(h);
  if (!T->factored) return -3;
  const long n = T->n;
  HCtx HL{T, &T->L, T->eps};
  HCtx HC{T, &T->C, T->eps};
  double logdet = 0.0;
  std::vector<int> lv;
  leaf_list(T->L, 0, lv);
  for (int b : lv) {
    const Block& bl = T->L[b];
    if (bl.diag)
      for (long i = 0; i < bl.D.m; ++i) logdet += 2.0 * std::log(bl.D(i, i));
  }
  auto dot = [n](const std::vector<double>& a, const std::vector<double>& b) {
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
  };
  auto precond = [&](std::vector<double>& v) {  // v := (L L^T)^-1 v
    trsv(HL, 0, View{v.data(), n, 1, n});
    trsv_t(HL, 0, View{v.data(), n, 1, n});
  };
  auto apply_C = [&](const std::vector<double>& x, std::vector<double>& y) {
    std::fill(y.begin(), y.end(), 0.0);
    symv(HC, 0, View{const_cast<double*>(x.data()), n, 1, n}, View{y.data(), n, 1, n});
  };
  std::vector<double> zt(n);
  for (long i = 0; i < n; ++i) zt[i] = z[T->perm[i]];
  // eq. (2): v = L^-1 z, quad_factor = v^T v
  std::vector<double> v = zt;
  trsv(HL, 0, View{v.data(), n, 1, n});
  const double qf = dot(v, v);
  // PCG with x0 = (L L^T)^-1 z
  std::vector<double> x = v;
  trsv_t(HL, 0, View{x.data(), n, 1, n});
  std::vector<double> r(n), q(n), p(n), w(n);
  apply_C(x, q);
  for (long i = 0; i < n; ++i) r[i] = zt[i] - q[i];
  const double zn = std::sqrt(dot(zt, zt));
  double rel = zn > 0.0 ? std::sqrt(dot(r, r)) / zn : 0.0;
  int it = 0;
  if (rel > tol) {
    w = r;
    precond(w);
    p = w;
    double rw = dot(r, w);
    while (it < maxit) {
      apply_C(p, q);
      const double alpha = rw / dot(p, q);
      for (long i = 0; i < n; ++i) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
      }
      ++it;
      rel = zn > 0.0 ? std::sqrt(dot(r, r)) / zn : 0.0;
      if (rel <= tol) break;
      w = r;
      precond(w);
      const double rw1 = dot(r, w);
      const double beta = rw1 / rw;
      rw = rw1;
      for (long i = 0; i < n; ++i) p[i] = w[i] + beta * p[i];
    }
  }
  // true residual at exit
  apply_C(x, q);
  double rn = 0.0;
  for (long i = 0; i < n; ++i) rn += (zt[i] - q[i]) * (zt[i] - q[i]);
  rel = zn > 0.0 ? std::sqrt(rn) / zn : 0.0;
  const double quad = dot(zt, x);
  out[0] = -0.5 * n * std::log(2.0 * M_PI) - 0.5 * logdet - 0.5 * quad;
  out[1] = logdet;
  out[2] = quad;
  out[3] = qf;
  out[4] = it;
  out[5] = rel;
  return 0;
}

// Standalone pieces exposed for the pin tests.
// ACA + truncation of the block rows [r0, r0+m) x cols [c0, c0+n) of the
// current tree (after assemble set theta): returns rank, fills U (m x k), V.
long orc_h_aca_block(void* h, long r0, long m, long c0, long n, double eps, long kmax, double* U,
                     double* V, int recompress) {
  HTree* T = static_cast<HTree*>(h);
  Mat Um, Vm;
  aca(*T, r0, m, c0, n, eps, kmax, Um, Vm);
  if (recompress) truncate_lr(Um, Vm, eps);
  std::copy(Um.a.begin(), Um.a.end(), U);
  std::copy(Vm.a.begin(), Vm.a.end(), V);
  return Um.n;
}

// Truncation of U V^T (m x K, n x K) in place into the leading k columns.
long orc_truncate(double* U, long m, double* V, long n, long K, double eps) {
  Mat Um(m, K), Vm(n, K);
  std::copy(U, U + m * K, Um.a.begin());
  std::copy(V, V + n * K, Vm.a.begin());
  truncate_lr(Um, Vm, eps);
  std::copy(Um.a.begin(), Um.a.end(), U);
  std::copy(Vm.a.begin(), Vm.a.end(), V);
  return Um.n;
}

// Set theta without assembling (for orc_h_aca_block).
// Fixed-rank mode (Tables 2 and 3): every low-rank block -- ACA and every
// truncation -- keeps at most k columns; k = 0 restores the adaptive rank.
int orc_h_set_fixed_rank(void* h, long k) {
  if (k < 0) return -1;
  static_cast<HTree*>(h)->kfix = k;
  return 0;
}

int orc_h_set_theta(void* h, double sigma2, double ell, double nu, double nugget) {
  HTree* T = static_cast<HTree*>(h);
  T->th = Theta{sigma2, ell, nu, nugget};
  return 0;
}

}  // extern "C"
