// Host setup: open knot vectors, B-spline derivatives on the non-zero span,
// Greville collocation points, banded collocation factors, and the FD eigen-
// factors of each direction (computed with cuSOLVER on the device, FP64).
//
// Paper: Sec. 2.1 (open knots, basis), Sec. 2.2 eq. (greville) and
// eq. (univariatecolloc) (M = B(tau), K = -B''(tau)), Sec. 4 eq. (eigendecomposition)
// and V := (M U)^{-T}; Remark 1 (real spectrum, well-conditioned U) is checked.
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>

#include "iga_internal.h"

namespace iga {

// ------------------------------------------------------------------ basis (host)
// Span index mu (0-based knot index) with t[mu] <= x < t[mu+1], p <= mu <= m-1;
// the right end x = t[m] belongs to the last span.
int find_span(const std::vector<double> &t, int p, int m, double x) {
  if (x >= t[m]) return m - 1;
  int lo = p, hi = m;  // invariant: t[lo] <= x < t[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (x < t[mid]) hi = mid; else lo = mid;
  }
  return lo;
}

// Values and first/second derivatives of the p+1 functions B_{mu-p..mu} that are
// non-zero on span mu.  tab[q][r] holds B_{mu-q+r, q}(x) for degrees q <= p built
// by the two-term recursion; derivatives of degree-p functions follow from the
// derivative identity D B_{i,q} = q (B_{i,q-1}/(t_{i+q}-t_i) - B_{i+1,q-1}/(t_{i+q+1}-t_{i+1})),
// applied once (D) or twice (D^2, through degree q-1 derivatives).
void span_basis(const std::vector<double> &t, int p, int mu, double x,
                double out[3][kMaxBand]) {
  double tab[kMaxDeg + 1][kMaxBand] = {};
  tab[0][0] = 1.0;
  for (int q = 1; q <= p; ++q) {
    for (int r = 0; r <= q; ++r) {
      const int i = mu - q + r;
      double v = 0.0;
      if (r >= 1) {  // B_{i,q-1} = tab[q-1][r-1]
        const double den = t[i + q] - t[i];
        if (den > 0.0) v += (x - t[i]) / den * tab[q - 1][r - 1];
      }
      if (r <= q - 1) {  // B_{i+1,q-1} = tab[q-1][r]
        const double den = t[i + q + 1] - t[i + 1];
        if (den > 0.0) v += (t[i + q + 1] - x) / den * tab[q - 1][r];
      }
      tab[q][r] = v;
    }
  }
  // D of degree-q functions from degree q-1 values: d1[q][r] for B_{mu-q+r,q}.
  auto deriv_from = [&](const double *low, int q, double *dst) {
    for (int r = 0; r <= q; ++r) {
      const int i = mu - q + r;
      double v = 0.0;
      if (r >= 1) {
        const double den = t[i + q] - t[i];
        if (den > 0.0) v += q * low[r - 1] / den;
      }
      if (r <= q - 1) {
        const double den = t[i + q + 1] - t[i + 1];
        if (den > 0.0) v -= q * low[r] / den;
      }
      dst[r] = v;
    }
  };
  double d1p[kMaxBand] = {}, d1pm1[kMaxBand] = {}, d2p[kMaxBand] = {};
  deriv_from(tab[p - 1], p, d1p);
  if (p >= 2) {
    deriv_from(tab[p - 2], p - 1, d1pm1);
    deriv_from(d1pm1, p, d2p);
  }
  for (int r = 0; r <= p; ++r) {
    out[0][r] = tab[p][r];
    out[1][r] = d1p[r];
    out[2][r] = d2p[r];
  }
}

void build_basis_1d(Factor1D &f) {
  const int p = f.p, ne = f.n_elem;
  const int m = ne + p;
  f.n = m - 2;
  f.W = p + 1;
  f.knots.assign(m + p + 1, 0.0);
  for (int k = 0; k < ne - 1; ++k) f.knots[p + 1 + k] = double(k + 1) / double(ne);
  for (int k = 0; k <= p; ++k) f.knots[m + k] = 1.0;
  // eq. (greville): tau_i = (1/p) sum_{j=1..p} xi_{i+j+1}, 1-based xi = t[.-1]
  f.tau.resize(f.n);
  for (int i = 1; i <= f.n; ++i) {
    double s = 0.0;
    for (int j = 1; j <= p; ++j) s += f.knots[i + j];
    f.tau[i - 1] = s / p;
  }
  const int n = f.n, W = f.W;
  f.start.assign(n, 0);
  for (int o = 0; o < 3; ++o) f.band[o].assign((size_t)n * W, 0.0);
  for (int i = 0; i < n; ++i) {
    const double x = f.tau[i];
    const int mu = find_span(f.knots, p, m, x);
    double vals[3][kMaxBand];
    span_basis(f.knots, p, mu, x, vals);
    // basis index b = mu - p + r; interior column j = b - 1 in [0, n)
    int st = mu - p - 1;
    st = std::max(0, std::min(st, n - W));
    f.start[i] = st;
    for (int r = 0; r <= p; ++r) {
      const int j = mu - p + r - 1;
      if (j < 0 || j >= n) continue;  // dropped boundary function (eq. space)
      const int tpos = j - st;
      for (int o = 0; o < 3; ++o) f.band[o][(size_t)i * W + tpos] = vals[o][r];
    }
  }
}

// ------------------------------------------------------------------ eigen-factors
#define CUSOLVER_TRY(expr)                                                          \
  do {                                                                              \
    cusolverStatus_t s_ = (expr);                                                   \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                              \
      throw Error{IGA_ERR_CUDA, std::string(#expr) + " failed with status " + std::to_string((int)s_)}; \
  } while (0)

namespace {
struct SolverHandle {
  cusolverDnHandle_t h = nullptr;
  cusolverDnParams_t prm = nullptr;
};

// One cuSOLVER handle per host thread and device, created on the thread's first
// eigensolve there and kept for the life of the process (never destroyed: destroying one
// frees device memory with a device-wide synchronisation, and at process exit the context
// may already be gone).  Created and used with the device lock held shared.
SolverHandle &thread_solver(cudaStream_t stream) {
  thread_local SolverHandle hs[64];
  int dev = 0;
  IGA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw Error{IGA_ERR_CUDA, "device index out of range"};
  SolverHandle &sh = hs[dev];
  if (!sh.h) {
    CUSOLVER_TRY(cusolverDnCreate(&sh.h));
    CUSOLVER_TRY(cusolverDnCreateParams(&sh.prm));
  }
  CUSOLVER_TRY(cusolverDnSetStream(sh.h, stream));
  return sh;
}

// Stream-ordered temporary device buffer of the eigensolves: cudaMallocAsync / cudaFreeAsync
// on the setup's own stream, so that freeing it does not synchronise the whole device (a
// cudaFree waits for every stream's work, the other setup threads' and the running solves').
template <class T> struct StreamBuf {
  T *ptr = nullptr;
  cudaStream_t s;
  StreamBuf(size_t n, cudaStream_t s_) : s(s_) {
    if (cudaMallocAsync((void **)&ptr, std::max<size_t>(n, 1) * sizeof(T), s) != cudaSuccess) {
      ptr = nullptr;
      (void)cudaGetLastError();
      throw Error{IGA_ERR_OOM, "cudaMallocAsync of " + std::to_string(n * sizeof(T)) + " bytes failed"};
    }
  }
  StreamBuf(const StreamBuf &) = delete;
  StreamBuf &operator=(const StreamBuf &) = delete;
  ~StreamBuf() {
    if (ptr) cudaFreeAsync(ptr, s);
  }
};

// largest singular value of a dense row-major n x n matrix by power iteration on A^T A
double norm2_est(const std::vector<double> &A, int n) {
  std::vector<double> x(n, 1.0 / std::sqrt((double)n)), y(n), z(n);
  double s = 0.0, s_prev = -1.0;
  // the estimate feeds only the cond(U) <= 1e3 check (Remark 1): six digits are plenty
  for (int it = 0; it < 60 && std::fabs(s - s_prev) > 1e-6 * s; ++it) {
    s_prev = s;
    for (int i = 0; i < n; ++i) {
      double a = 0.0;
      for (int j = 0; j < n; ++j) a += A[(size_t)i * n + j] * x[j];
      y[i] = a;
    }
    std::fill(z.begin(), z.end(), 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) z[j] += A[(size_t)i * n + j] * y[i];
    double nz = 0.0;
    for (double v : z) nz += v * v;
    nz = std::sqrt(nz);
    if (nz == 0.0) return 0.0;
    s = std::sqrt(nz);
    for (int j = 0; j < n; ++j) x[j] = z[j] / nz;
  }
  return s;
}
}  // namespace

// Real eigenpairs of the m x m pencil (K, M) (column-major): A = M^{-1} K by LU,
// then the eigenvalues and right eigenvectors of A.  Throws NOT_DIAGONALIZABLE for
// complex eigenvalues (Remark 1).  lam: m values; U: m x m column-major.
static void eig_pencil(SolverHandle &sh, const std::vector<double> &Kc,
                       const std::vector<double> &Mc, int m, std::vector<double> &lam,
                       std::vector<double> &U, cudaStream_t stream) {
  StreamBuf<double> dM((size_t)m * m, stream), dA((size_t)m * m, stream),
      dVR((size_t)m * m, stream), dW(2 * (size_t)m, stream);
  StreamBuf<int64_t> dipiv(m, stream);
  StreamBuf<int> dinfo(1, stream);
  IGA_CUDA_TRY(cudaMemcpyAsync(dM.ptr, Mc.data(), Mc.size() * 8, cudaMemcpyHostToDevice, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(dA.ptr, Kc.data(), Kc.size() * 8, cudaMemcpyHostToDevice, stream));
  auto check_info = [&](const char *what) {
    int info = 0;
    IGA_CUDA_TRY(cudaMemcpyAsync(&info, dinfo.ptr, sizeof(int), cudaMemcpyDeviceToHost, stream));
    IGA_CUDA_TRY(cudaStreamSynchronize(stream));
    if (info != 0)
      throw Error{IGA_ERR_NOT_DIAGONALIZABLE, std::string(what) + " info=" + std::to_string(info)};
  };
  size_t dws = 0, hws = 0;
  CUSOLVER_TRY(cusolverDnXgetrf_bufferSize(sh.h, sh.prm, m, m, CUDA_R_64F, dM.ptr, m, CUDA_R_64F,
                                           &dws, &hws));
  {
    StreamBuf<char> dbuf(std::max<size_t>(dws, 1), stream);
    std::vector<char> hbuf(std::max<size_t>(hws, 1));
    CUSOLVER_TRY(cusolverDnXgetrf(sh.h, sh.prm, m, m, CUDA_R_64F, dM.ptr, m, dipiv.ptr, CUDA_R_64F,
                                  dbuf.ptr, dws, hbuf.data(), hws, dinfo.ptr));
    check_info("getrf(M)");
  }
  CUSOLVER_TRY(cusolverDnXgetrs(sh.h, sh.prm, CUBLAS_OP_N, m, m, CUDA_R_64F, dM.ptr, m, dipiv.ptr,
                                CUDA_R_64F, dA.ptr, m, dinfo.ptr));
  check_info("getrs(M, K)");
  CUSOLVER_TRY(cusolverDnXgeev_bufferSize(sh.h, sh.prm, CUSOLVER_EIG_MODE_NOVECTOR,
                                          CUSOLVER_EIG_MODE_VECTOR, m, CUDA_R_64F, dA.ptr, m,
                                          CUDA_C_64F, dW.ptr, CUDA_R_64F, nullptr, 1, CUDA_R_64F,
                                          dVR.ptr, m, CUDA_R_64F, &dws, &hws));
  {
    StreamBuf<char> dbuf(std::max<size_t>(dws, 1), stream);
    std::vector<char> hbuf(std::max<size_t>(hws, 1));
    CUSOLVER_TRY(cusolverDnXgeev(sh.h, sh.prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR,
                                 m, CUDA_R_64F, dA.ptr, m, CUDA_C_64F, dW.ptr, CUDA_R_64F, nullptr,
                                 1, CUDA_R_64F, dVR.ptr, m, CUDA_R_64F, dbuf.ptr, dws, hbuf.data(),
                                 hws, dinfo.ptr));
    check_info("geev(M^{-1}K)");
  }
  std::vector<double> Wc(2 * (size_t)m);
  U.resize((size_t)m * m);
  IGA_CUDA_TRY(cudaMemcpyAsync(Wc.data(), dW.ptr, Wc.size() * 8, cudaMemcpyDeviceToHost, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(U.data(), dVR.ptr, U.size() * 8, cudaMemcpyDeviceToHost, stream));
  IGA_CUDA_TRY(cudaStreamSynchronize(stream));
  lam.resize(m);
  for (int j = 0; j < m; ++j) {
    const double re = Wc[2 * j], im = Wc[2 * j + 1];
    const double mag = std::sqrt(re * re + im * im);
    if (!std::isfinite(mag) || std::fabs(im) > 1e-10 * std::max(mag, 1e-300))
      throw Error{IGA_ERR_NOT_DIAGONALIZABLE, "complex eigenvalue of M^{-1}K (Remark 1)"};
    lam[j] = re;
  }
}

static bool reflection_symmetric(const std::vector<double> &A, int n) {
  double mx = 0.0, diff = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double a = A[i + (size_t)n * j];
      mx = std::max(mx, std::fabs(a));
      diff = std::max(diff, std::fabs(A[(n - 1 - i) + (size_t)n * (n - 1 - j)] - a));
    }
  return diff <= 1e-12 * mx;
}

// Eigenvectors as columns of an n x n column-major matrix and eigenvalues (unsorted).
// On uniform knots the factors commute with the flip i -> n-1-i, so the pencil is
// solved separately on the even subspace (v_i = v_{n-1-i}) and the odd subspace
// (v_i = -v_{n-1-i}); Remark 1's double outlier eigenvalue then has one eigenvector
// in each half and U stays well conditioned.
static void eig_all(SolverHandle &sh, const std::vector<double> &Kc, const std::vector<double> &Mc,
                    int n, std::vector<double> &lam, std::vector<double> &Ucol,
                    cudaStream_t stream) {
  if (!(reflection_symmetric(Kc, n) && reflection_symmetric(Mc, n))) {
    eig_pencil(sh, Kc, Mc, n, lam, Ucol, stream);
    return;
  }
  const int h = n / 2, ne = h + n % 2, no = h;
  const double c = 1.0 / std::sqrt(2.0);
  // basis column q of the even (sgn=+1) / odd (sgn=-1) subspace, as (index, weight) pairs
  auto basis = [&](int q, int sgn, int *idx, double *wt) -> int {
    if (q < h) {
      idx[0] = q;
      wt[0] = c;
      idx[1] = n - 1 - q;
      wt[1] = sgn * c;
      return 2;
    }
    idx[0] = h;  // middle entry (n odd, even part only)
    wt[0] = 1.0;
    return 1;
  };
  lam.clear();
  Ucol.assign((size_t)n * n, 0.0);
  int col = 0;
  for (int part = 0; part < 2; ++part) {
    const int m = part == 0 ? ne : no, sgn = part == 0 ? 1 : -1;
    if (m == 0) continue;
    std::vector<double> Kq((size_t)m * m), Mq((size_t)m * m);
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b) {
        int ia[2], ib[2];
        double wa[2], wb[2];
        const int na = basis(a, sgn, ia, wa), nb = basis(b, sgn, ib, wb);
        double sk = 0.0, sm = 0.0;
        for (int u = 0; u < na; ++u)
          for (int v = 0; v < nb; ++v) {
            sk += wa[u] * wb[v] * Kc[ia[u] + (size_t)n * ib[v]];
            sm += wa[u] * wb[v] * Mc[ia[u] + (size_t)n * ib[v]];
          }
        Kq[a + (size_t)m * b] = sk;
        Mq[a + (size_t)m * b] = sm;
      }
    std::vector<double> lq, Uq;
    eig_pencil(sh, Kq, Mq, m, lq, Uq, stream);
    for (int j = 0; j < m; ++j, ++col) {
      lam.push_back(lq[j]);
      for (int a = 0; a < m; ++a) {
        int ia[2];
        double wa[2];
        const int na = basis(a, sgn, ia, wa);
        for (int u = 0; u < na; ++u) Ucol[ia[u] + (size_t)n * col] += wa[u] * Uq[a + (size_t)m * j];
      }
    }
  }
}

static void eigen_factors(Factor1D &f, cudaStream_t stream) {
  const int n = f.n;
  // the FD pencil (K, M) as bands: the collocation factors of eq. (univariatecolloc)
  // (K + shift B' for a wind, Sec. 3.2), or the WQ Galerkin factors of eq. (univariateWQ)
  const bool gal = f.scheme == 1;
  const int W = gal ? f.GW : f.W;
  auto mstart = [&](int i) { return gal ? f.gstart[i] : f.start[i]; };
  auto mval = [&](int i, int t) {
    return gal ? f.gM[(size_t)i * W + t] : f.band[0][(size_t)i * W + t];
  };
  auto kval = [&](int i, int t) {
    return gal ? f.gK[(size_t)i * W + t]
               : -f.band[2][(size_t)i * W + t] + f.shift * f.band[1][(size_t)i * W + t];
  };
  // dense column-major M and K
  std::vector<double> Mc((size_t)n * n, 0.0), Kc((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int t = 0; t < W; ++t) {
      const int j = mstart(i) + t;
      Mc[i + (size_t)n * j] = mval(i, t);
      Kc[i + (size_t)n * j] = kval(i, t);
    }
  // Every CUDA and cuSOLVER call of this function -- the thread's handle creation on its
  // first use (which may load library code), allocations, frees, solves -- runs with the
  // device lock held shared; the O(n^2 W) host work between them runs unlocked.
  std::vector<double> lam_u, VR;
  const double ts0 = wall_seconds();
  std::shared_lock<DeviceLock> dlk(device_mutex());
  SolverHandle *sh = &thread_solver(stream);
  eig_all(*sh, Kc, Mc, n, lam_u, VR, stream);
  dlk.unlock();
  f.setup_solver_s = wall_seconds() - ts0;
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam_u[a] < lam_u[b]; });
  f.lam.resize(n);
  f.U.assign((size_t)n * n, 0.0);
  for (int jj = 0; jj < n; ++jj) {
    const int j = order[jj];
    f.lam[jj] = lam_u[j];
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) nrm += VR[i + (size_t)n * j] * VR[i + (size_t)n * j];
    nrm = std::sqrt(nrm);
    for (int i = 0; i < n; ++i) f.U[(size_t)i * n + jj] = VR[i + (size_t)n * j] / nrm;
  }
  // MU (banded M times dense U), then V^T = (M U)^{-1}
  std::vector<double> MUc((size_t)n * n, 0.0), Ic((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int t = 0; t < W; ++t) {
      const double mv = mval(i, t);
      if (mv == 0.0) continue;
      const int k = mstart(i) + t;
      for (int j = 0; j < n; ++j) MUc[i + (size_t)n * j] += mv * f.U[(size_t)k * n + j];
    }
  for (int i = 0; i < n; ++i) Ic[i + (size_t)n * i] = 1.0;
  std::vector<double> Xc((size_t)n * n);
  const double ts1 = wall_seconds();
  dlk.lock();
  {  // the buffers are freed (stream-ordered) before the lock is released
    sh = &thread_solver(stream);
    StreamBuf<double> dM((size_t)n * n, stream), dX((size_t)n * n, stream);
    StreamBuf<int64_t> dipiv(n, stream);
    StreamBuf<int> dinfo(1, stream);
    auto check_info = [&](const char *what) {
      int info = 0;
      IGA_CUDA_TRY(cudaMemcpyAsync(&info, dinfo.ptr, sizeof(int), cudaMemcpyDeviceToHost, stream));
      IGA_CUDA_TRY(cudaStreamSynchronize(stream));
      if (info != 0)
        throw Error{IGA_ERR_NOT_DIAGONALIZABLE, std::string(what) + " info=" + std::to_string(info)};
    };
    size_t dws = 0, hws = 0;
    IGA_CUDA_TRY(cudaMemcpyAsync(dM.ptr, MUc.data(), MUc.size() * 8, cudaMemcpyHostToDevice, stream));
    IGA_CUDA_TRY(cudaMemcpyAsync(dX.ptr, Ic.data(), Ic.size() * 8, cudaMemcpyHostToDevice, stream));
    CUSOLVER_TRY(cusolverDnXgetrf_bufferSize(sh->h, sh->prm, n, n, CUDA_R_64F, dM.ptr, n, CUDA_R_64F,
                                             &dws, &hws));
    {
      StreamBuf<char> dbuf(std::max<size_t>(dws, 1), stream);
      std::vector<char> hbuf(std::max<size_t>(hws, 1));
      CUSOLVER_TRY(cusolverDnXgetrf(sh->h, sh->prm, n, n, CUDA_R_64F, dM.ptr, n, dipiv.ptr, CUDA_R_64F,
                                    dbuf.ptr, dws, hbuf.data(), hws, dinfo.ptr));
      check_info("getrf(MU)");
    }
    CUSOLVER_TRY(cusolverDnXgetrs(sh->h, sh->prm, CUBLAS_OP_N, n, n, CUDA_R_64F, dM.ptr, n, dipiv.ptr,
                                  CUDA_R_64F, dX.ptr, n, dinfo.ptr));
    check_info("getrs(MU, I)");
    IGA_CUDA_TRY(cudaMemcpyAsync(Xc.data(), dX.ptr, Xc.size() * 8, cudaMemcpyDeviceToHost, stream));
    IGA_CUDA_TRY(cudaStreamSynchronize(stream));
  }
  dlk.unlock();
  f.setup_solver_s += wall_seconds() - ts1;
  f.Vt.resize((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) f.Vt[(size_t)i * n + j] = Xc[i + (size_t)n * j];
  // Remark 1: cond_2(U) = ||U|| ||U^{-1}||, with U^{-1} = V^T M
  std::vector<double> Uinv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int r = 0; r < n; ++r) {
      const double a = f.Vt[(size_t)i * n + r];
      for (int t = 0; t < W; ++t) Uinv[(size_t)i * n + mstart(r) + t] += a * mval(r, t);
    }
  f.cond_U = norm2_est(f.U, n) * norm2_est(Uinv, n);
  if (!(f.cond_U <= 1e3))
    throw Error{IGA_ERR_NOT_DIAGONALIZABLE,
                "ill-conditioned eigenvector matrix, cond(U) ~ " + std::to_string(f.cond_U)};
}

// ------------------------------------------------------------------ device upload
template <class T> static void upload(DevBuf<T> &d, const std::vector<T> &h, cudaStream_t s) {
  d.alloc(h.size());
  IGA_CUDA_TRY(cudaMemcpyAsync(d.ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

// FP32 value rounded to the nearest TF32 (10-bit mantissa), ties to even.
static float to_tf32(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) {
    u += 0xfffu + ((u >> 13) & 1u);
    u &= ~0x1fffu;
  }
  std::memcpy(&x, &u, 4);
  return x;
}

// Folded FD factors.  Each eigenvector u_j is even (u_{n-1-i} = u_i) or odd
// (u_{n-1-i} = -u_i) when the pencil was solved on its reflection halves; then V^T and
// U are block diagonal in the basis of sums / differences of mirrored entries, and the
// blocks are the left halves of their rows.  Order the eigen-index [even | odd] (by
// eigenvalue within each part):
//   Bf[c][f] (forward):  even c: Vt[j][f] for f < ne (f = h is the middle entry);
//                        odd c:  Vt[j][a] at f = ne + a, a < h;          j = perm[c]
//   Bi[a][k] (inverse):  U[a][perm[k]] for a < ne, and 0 for odd k at the middle row.
// Left unset (dense products used) when some eigenvector has no parity.
static void build_folded(Factor1D &f, cudaStream_t s) {
  const int n = f.n, h = n / 2;
  std::vector<int> even, odd;
  for (int j = 0; j < n; ++j) {
    double par = 0.0;
    for (int i = 0; i < n; ++i) par += f.U[(size_t)i * n + j] * f.U[(size_t)(n - 1 - i) * n + j];
    if (std::fabs(par - 1.0) < 1e-9) even.push_back(j);
    else if (std::fabs(par + 1.0) < 1e-9) odd.push_back(j);
    else return;
  }
  const int ne = (int)even.size();
  if (ne != h + n % 2 || (int)odd.size() != h) return;
  std::vector<int> perm(even);
  perm.insert(perm.end(), odd.begin(), odd.end());
  std::vector<double> Bf((size_t)n * n, 0.0), Bi((size_t)ne * n, 0.0), lamf(n);
  for (int c = 0; c < n; ++c) {
    const int j = perm[c];
    lamf[c] = f.lam[j];
    if (c < ne) {
      for (int q = 0; q < ne; ++q) Bf[(size_t)c * n + q] = f.Vt[(size_t)j * n + q];
    } else {
      for (int a = 0; a < h; ++a) Bf[(size_t)c * n + ne + a] = f.Vt[(size_t)j * n + a];
    }
  }
  for (int a = 0; a < ne; ++a)
    for (int k = 0; k < n; ++k)
      if (k < ne || a < h) Bi[(size_t)a * n + k] = f.U[(size_t)a * n + perm[k]];
  std::vector<double> BfT((size_t)n * n), BiT((size_t)n * ne);
  for (int c = 0; c < n; ++c)
    for (int q = 0; q < n; ++q) BfT[(size_t)q * n + c] = Bf[(size_t)c * n + q];
  for (int a = 0; a < ne; ++a)
    for (int k = 0; k < n; ++k) BiT[(size_t)k * ne + a] = Bi[(size_t)a * n + k];
  upload(f.d_Bf, Bf, s);
  upload(f.d_Bi, Bi, s);
  upload(f.d_BfT, BfT, s);
  upload(f.d_BiT, BiT, s);
  upload(f.d_lam_fold, lamf, s);
  f.ne = ne;
  f.folded = true;
}

static void upload_factor(Factor1D &f, cudaStream_t s) {
  upload(f.d_start, f.start, s);
  for (int o = 0; o < 3; ++o) upload(f.d_band[o], f.band[o], s);
  upload(f.d_tau, f.tau, s);
  upload(f.d_lam, f.lam, s);
  upload(f.d_Vt, f.Vt, s);
  upload(f.d_U, f.U, s);
  // tensor-core operands: row-major, leading dimension padded to a multiple of 8
  const int n = f.n;
  f.kpad = (n + 7) / 8 * 8;
  std::vector<float> vt32((size_t)n * f.kpad, 0.f), u32((size_t)n * f.kpad, 0.f);
  std::vector<float> vt32lo((size_t)n * f.kpad, 0.f), u32lo((size_t)n * f.kpad, 0.f);
  std::vector<__nv_bfloat16> vt16((size_t)n * f.kpad, __float2bfloat16(0.f)),
      u16((size_t)n * f.kpad, __float2bfloat16(0.f));
  // TF32 part and the TF32 rounding of the remainder (error-compensated TF32 form)
  auto split = [](double v, float &hi, float &lo) {
    hi = to_tf32((float)v);
    lo = to_tf32((float)(v - (double)hi));
  };
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const size_t o = (size_t)i * f.kpad + j;
      split(f.Vt[(size_t)i * n + j], vt32[o], vt32lo[o]);
      split(f.U[(size_t)i * n + j], u32[o], u32lo[o]);
      vt16[o] = __float2bfloat16((float)f.Vt[(size_t)i * n + j]);
      u16[o] = __float2bfloat16((float)f.U[(size_t)i * n + j]);
    }
  upload(f.d_Vt32, vt32, s);
  upload(f.d_U32, u32, s);
  upload(f.d_Vt32lo, vt32lo, s);
  upload(f.d_U32lo, u32lo, s);
  upload(f.d_Vt16, vt16, s);
  upload(f.d_U16, u16, s);
  if (f.scheme == 1) {
    upload(f.d_xq, f.xq, s);
    upload(f.d_qstart, f.qstart, s);
    upload(f.d_wstart, f.wstart, s);
    for (int b = 0; b < 2; ++b) upload(f.d_qband[b], f.qband[b], s);
    for (int k = 0; k < 4; ++k) upload(f.d_wband[k], f.wband[k], s);
  }
  build_folded(f, s);
  IGA_CUDA_TRY(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ device-wide lock
DeviceLock &device_mutex() {
  static DeviceLock mu;
  return mu;
}

int verbose_level() {
  static const int v = [] {
    const char *e = std::getenv("IGA_VERBOSE");
    return e ? std::atoi(e) : 0;
  }();
  return v;
}

double wall_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

int pdl_mask() {
  // measured on GB300 (3D n = 65 solves): programmatic dependent launch pays off for
  // the FD mode products (FP64 and tensor-core chains), is neutral for the operator
  // passes and costs ~0.7 ms per solve for the Krylov reductions, whose early-scheduled
  // waiting blocks slow the last-block reductions down
  static const int mask = [] {
    const char *e = std::getenv("IGA_PDL");
    return e ? std::atoi(e) : (int)(kPdlFd64 | kPdlTensorCore);
  }();
  return mask;
}


void ensure_kernels_loaded() {
  static std::atomic<bool> loaded[64] = {};
  int dev = 0;
  IGA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && loaded[dev].load(std::memory_order_acquire)) return;
  std::unique_lock<DeviceLock> lk(device_mutex());
  if (dev < 0 || dev >= 64 || loaded[dev].load(std::memory_order_relaxed)) return;
  preload_kernels_fd64();
  preload_kernels_fd64_fma();
  preload_kernels_fd_tc();
  preload_kernels_fd_f64tc();
  preload_kernels_geom_op();
  preload_kernels_krylov();
  preload_kernels_bicgstab();
  preload_kernels_wq();
  loaded[dev].store(true, std::memory_order_release);
}

// ------------------------------------------------------------------ factor cache
std::shared_ptr<Factor1D> get_factor(int n_elem, int p, cudaStream_t stream, double shift,
                                     int scheme) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, long long, int>, std::weak_ptr<Factor1D>> cache;
  int dev = 0;
  IGA_CUDA_TRY(cudaGetDevice(&dev));
  long long sbits = 0;
  std::memcpy(&sbits, &shift, sizeof(sbits));
  const auto key = std::make_tuple(dev, n_elem, p, sbits, scheme);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      if (auto sp = it->second.lock()) return sp;
    }
  }
  // computed without the lock so that setups of different shapes on different host
  // threads overlap; if two threads race on one shape, the first to publish wins
  auto f = std::make_shared<Factor1D>();
  f->n_elem = n_elem;
  f->p = p;
  f->shift = shift;
  f->scheme = scheme;
  const double t0 = wall_seconds();
  build_basis_1d(*f);
  if (scheme == 1) build_wq_1d(*f);
  const double t1 = wall_seconds();
  eigen_factors(*f, stream);
  const double t2 = wall_seconds();
  upload_factor(*f, stream);
  if (verbose_level() >= 2)
    std::fprintf(stderr, "iga setup n_elem=%d p=%d: 1D basis %.1f ms, eigen-factors %.1f ms "
                 "(cuSOLVER with the lock wait %.1f ms), upload %.1f ms\n", n_elem, p,
                 1e3 * (t1 - t0), 1e3 * (t2 - t1), 1e3 * f->setup_solver_s,
                 1e3 * (wall_seconds() - t2));
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) {
    if (auto sp = it->second.lock()) return sp;
  }
  cache[key] = f;
  return f;
}

// ------------------------------------------------------------------ fields
int num_fields(int d) { return d == 2 ? 5 : 9; }

FieldDesc field_desc(int d, int f) {
  FieldDesc fd{{0, 0, 0}};
  if (d == 2) {
    static const int o[5][2] = {{2, 0}, {0, 2}, {1, 1}, {1, 0}, {0, 1}};
    fd.order[0] = o[f][0];
    fd.order[1] = o[f][1];
  } else {
    static const int o[9][3] = {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1},
                                {0, 1, 1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int l = 0; l < 3; ++l) fd.order[l] = o[f][l];
  }
  return fd;
}

}  // namespace iga
