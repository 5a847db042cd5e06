// Weighted-quadrature (WQ) Galerkin discretization, univariate part (Sec. 2.3).
//
// A_wq of eq. (WQapprox) is a sum over (a, b) of tensor products of univariate
// operators: the trial functions' values or first derivatives at the quadrature points
// (B^{(t)}, nq x n) and univariate weighted-quadrature rules w^{(s,t)} (n x nq) that
// absorb the test function's value (s = 0) or derivative (s = 1).  A rule is fixed by
// exactness on the spline space (the construction the paper takes from Calabro,
// Sangalli and Tani 2017, with the readings below):
//   sum_q w^{(s,t)}_{i,q} B_j^{(t)}(x_q) = int_0^1 B_i^{(s)} B_j^{(t)} dx
// for every basis function B_j (full basis) whose support meets that of B_i; the
// weights of row i live on the quadrature points in the support of B_i and are the
// minimum 2-norm solution.  For t = 1 the conditions are linearly dependent (the
// derivatives of the overlapping functions sum to zero at every point of the support,
// and so do the right-hand sides), so the last condition is dropped; the remaining
// system has full row rank and the same minimum-norm solution.
// Quadrature points: every element end point and midpoint, and p equispaced interior
// points in the first and the last element.  The univariate Galerkin matrices
// M = int B_i B_j and K = int B_i' B_j' (eq. univariateWQ) are the FD pencil of
// P_wq (Sec. 3), symmetric positive definite (the symmetric FD of Sec. 4).
#include <algorithm>
#include <cmath>
#include <vector>

#include "iga_internal.h"

namespace iga {

// k-point Gauss-Legendre rule on [-1, 1].  The nodes are the roots of the Legendre
// polynomial P_k, found by Newton's method from cos(pi (i + 3/4) / (k + 1/2)); P_k and
// P_k' come from the recurrence j P_j = (2j - 1) x P_{j-1} - (j - 1) P_{j-2} and
// (x^2 - 1) P_k' = k (x P_k - P_{k-1}); the weights are 2 / ((1 - x^2) P_k'(x)^2).
static void gauss_legendre(int k, std::vector<double> &x, std::vector<double> &w) {
  x.assign(k, 0.0);
  w.assign(k, 0.0);
  for (int i = 0; i < k; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (k + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= k; ++j) {
        const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = k * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[k - 1 - i] = z;  // ascending
    w[k - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Minimum 2-norm solution of E w = r for a rows x cols matrix E (row-major) of full row
// rank, rows <= cols: Householder QR of E^T = Q R, then R^T z = r, w = Q z.
static void min_norm_solve(int rows, int cols, const std::vector<double> &E, const double *r,
                           double *w) {
  // A = E^T, cols x rows, column-major in a[j * cols + i]
  std::vector<double> a((size_t)rows * cols), v((size_t)rows * cols, 0.0), diag(rows);
  for (int i = 0; i < rows; ++i)
    for (int j = 0; j < cols; ++j) a[(size_t)i * cols + j] = E[(size_t)i * cols + j];
  double scale = 0.0;
  for (double x : a) scale = std::max(scale, std::fabs(x));
  for (int k = 0; k < rows; ++k) {
    double *col = &a[(size_t)k * cols];
    double nrm = 0.0;
    for (int i = k; i < cols; ++i) nrm += col[i] * col[i];
    nrm = std::sqrt(nrm);
    if (!(nrm > 1e-13 * scale))
      throw Error{IGA_ERR_INVALID_ARG, "weighted-quadrature rule: singular exactness system"};
    const double alpha = col[k] > 0.0 ? -nrm : nrm;
    double *vk = &v[(size_t)k * cols];
    for (int i = k; i < cols; ++i) vk[i] = col[i];
    vk[k] -= alpha;
    double vv = 0.0;
    for (int i = k; i < cols; ++i) vv += vk[i] * vk[i];
    diag[k] = alpha;
    for (int j = k + 1; j < rows; ++j) {  // apply H_k to the later columns
      double *cj = &a[(size_t)j * cols];
      double s = 0.0;
      for (int i = k; i < cols; ++i) s += vk[i] * cj[i];
      s = 2.0 * s / vv;
      for (int i = k; i < cols; ++i) cj[i] -= s * vk[i];
    }
    for (int i = k; i < cols; ++i) vk[i] /= std::sqrt(vv);  // unit reflector
  }
  // R^T z = r: R[j][k] = a[k * cols + j] (j < k), R[k][k] = diag[k]
  std::vector<double> y(cols, 0.0);
  for (int k = 0; k < rows; ++k) {
    double s = r[k];
    for (int j = 0; j < k; ++j) s -= a[(size_t)k * cols + j] * y[j];
    y[k] = s / diag[k];
  }
  // w = H_0 .. H_{rows-1} [z; 0]
  for (int k = rows - 1; k >= 0; --k) {
    const double *vk = &v[(size_t)k * cols];
    double s = 0.0;
    for (int i = k; i < cols; ++i) s += vk[i] * y[i];
    for (int i = k; i < cols; ++i) y[i] -= 2.0 * s * vk[i];
  }
  for (int i = 0; i < cols; ++i) w[i] = y[i];
}

void build_wq_1d(Factor1D &f) {
  const int p = f.p, ne = f.n_elem, m = ne + p, n = m - 2, W = p + 1;
  const std::vector<double> &t = f.knots;
  // quadrature points
  std::vector<double> xs;
  for (int e = 0; e <= ne; ++e) xs.push_back(double(e) / double(ne));
  for (int e = 0; e < ne; ++e) {
    const double a = double(e) / double(ne), b = double(e + 1) / double(ne);
    if (e == 0 || e == ne - 1) {
      for (int u = 1; u <= p; ++u) xs.push_back(a + (b - a) * (double(u) / double(p + 1)));
    } else {
      xs.push_back(0.5 * (a + b));
    }
  }
  std::sort(xs.begin(), xs.end());
  xs.erase(std::unique(xs.begin(), xs.end()), xs.end());
  f.xq = xs;
  const int nq = f.nq = (int)xs.size();

  // univariate Galerkin integrals of the full basis, G[2 s + t][i m + j], by Gauss-Legendre
  // with p + 1 points per element (the integrand is a polynomial of degree <= 2p there)
  std::vector<double> G[4];
  for (auto &g : G) g.assign((size_t)m * m, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(p + 1, gx, gw);
  for (int e = 0; e < ne; ++e) {
    const double a = double(e) / double(ne), b = double(e + 1) / double(ne);
    const int mu = p + e;  // the span [t_mu, t_mu+1) of element e
    for (int g = 0; g <= p; ++g) {
      const double x = 0.5 * (b - a) * gx[g] + 0.5 * (a + b), wt = 0.5 * (b - a) * gw[g];
      double v[3][kMaxBand];
      span_basis(t, p, mu, x, v);
      for (int r1 = 0; r1 <= p; ++r1)
        for (int r2 = 0; r2 <= p; ++r2) {
          const size_t ij = (size_t)(mu - p + r1) * m + (mu - p + r2);
          for (int s = 0; s < 2; ++s)
            for (int tt = 0; tt < 2; ++tt) G[2 * s + tt][ij] += wt * v[s][r1] * v[tt][r2];
        }
    }
  }

  // full-basis values and derivatives at the quadrature points, and the interior bands
  std::vector<int> qmu(nq);
  std::vector<double> qv((size_t)nq * 2 * W);  // [q][b][r], function qmu[q] - p + r
  f.qstart.assign(nq, 0);
  for (int b = 0; b < 2; ++b) f.qband[b].assign((size_t)nq * W, 0.0);
  for (int q = 0; q < nq; ++q) {
    const int mu = find_span(t, p, m, xs[q]);
    double v[3][kMaxBand];
    span_basis(t, p, mu, xs[q], v);
    qmu[q] = mu;
    int st = std::max(0, std::min(mu - p - 1, n - W));
    f.qstart[q] = st;
    for (int r = 0; r <= p; ++r) {
      for (int b = 0; b < 2; ++b) qv[((size_t)q * 2 + b) * W + r] = v[b][r];
      const int j = mu - p + r - 1;  // interior index
      if (j < 0 || j >= n) continue;
      for (int b = 0; b < 2; ++b) f.qband[b][(size_t)q * W + (j - st)] = v[b][r];
    }
  }
  auto full_at = [&](int b, int j, int q) -> double {  // B_j^{(b)}(x_q), full basis
    const int r = j - (qmu[q] - p);
    return (r < 0 || r > p) ? 0.0 : qv[((size_t)q * 2 + b) * W + r];
  };

  // univariate rules of the interior test functions
  std::vector<int> q0(n), q1(n);
  int WW = 0;
  for (int i = 0; i < n; ++i) {
    const int I = i + 1;  // full-basis index
    const double lo = t[I], hi = t[I + p + 1];
    int a = 0;
    while (a < nq && xs[a] < lo) ++a;
    int b = a;
    while (b + 1 < nq && xs[b + 1] <= hi) ++b;
    q0[i] = a;
    q1[i] = b;
    WW = std::max(WW, b - a + 1);
  }
  f.WW = WW;
  f.wstart.assign(n, 0);
  for (int k = 0; k < 4; ++k) f.wband[k].assign((size_t)n * WW, 0.0);
  std::vector<double> E, rhs, w;
  for (int i = 0; i < n; ++i) {
    const int I = i + 1;
    const double lo = t[I], hi = t[I + p + 1];
    int j0 = 0;
    while (!(t[j0 + p + 1] > lo)) ++j0;
    int j1 = j0;
    while (j1 + 1 < m && t[j1 + 1] < hi) ++j1;
    const int npt = q1[i] - q0[i] + 1;
    const int st = std::min(q0[i], nq - WW);
    f.wstart[i] = st;
    for (int s = 0; s < 2; ++s)
      for (int tt = 0; tt < 2; ++tt) {
        const int rows = (j1 - j0 + 1) - tt;  // t = 1: one dependent condition dropped
        E.assign((size_t)rows * npt, 0.0);
        rhs.assign(rows, 0.0);
        w.assign(npt, 0.0);
        for (int c = 0; c < rows; ++c) {
          const int j = j0 + c;
          for (int u = 0; u < npt; ++u) E[(size_t)c * npt + u] = full_at(tt, j, q0[i] + u);
          rhs[c] = G[2 * s + tt][(size_t)I * m + j];
        }
        if (rows > npt)
          throw Error{IGA_ERR_INVALID_ARG, "weighted-quadrature rule: too few points"};
        min_norm_solve(rows, npt, E, rhs.data(), w.data());
        for (int u = 0; u < npt; ++u)
          f.wband[2 * s + tt][(size_t)i * WW + (q0[i] + u - st)] = w[u];
      }
  }

  // the Galerkin pencil (interior block), banded
  f.GW = 2 * p + 1;
  const int GW = std::min(f.GW, n);
  f.GW = GW;
  f.gstart.assign(n, 0);
  f.gM.assign((size_t)n * GW, 0.0);
  f.gK.assign((size_t)n * GW, 0.0);
  for (int i = 0; i < n; ++i) {
    const int st = std::max(0, std::min(i - p, n - GW));
    f.gstart[i] = st;
    for (int u = 0; u < GW; ++u) {
      const size_t ij = (size_t)(i + 1) * m + (st + u + 1);
      f.gM[(size_t)i * GW + u] = G[0][ij];
      f.gK[(size_t)i * GW + u] = G[3][ij];
    }
  }
}

}  // namespace iga
