// Geometry coefficients of the pulled-back operator and the matrix-free
// collocation operator by sum factorization (banded mode products).
//
// Operator (eq. collocation): (L u_h)(F(tau_I)) with L = -Lap and u_h = u_hat o F^{-1}.
// Pull-back: -Lap_x u = -sum_ab G^{ab} d_a d_b u_hat - sum_c L_c d_c u_hat with
// G = J^{-1} J^{-T}, L_c = -sum_k (J^{-1})_{ck} sum_ab G^{ab} d_a d_b F_k.
// Every derivative of u_hat at the tensor grid of collocation points is a tensor
// product of the 1D banded factors M = B(tau), B'(tau), B''(tau) (eq. univariatecolloc),
// applied mode by mode (sum factorization); the contraction with the fields is pointwise.
#include <cmath>

#include "fp_widen.h"
#include "contract_point.cuh"
#include "iga_internal.h"

namespace iga {

// ------------------------------------------------------------------ geometry
struct Geo3 {
  double J[3][3];
  double H[3][3][3];  // H[k][a][b] = d_a d_b F_k
};

__device__ static void ring_jh(double r0, double r1, double xi, double eta, double J[2][2],
                               double H[2][2][2], double *X) {
  const double R = r1 - r0, r = r0 + R * xi, w = 0.5 * M_PI, th = w * eta;
  double s, c;
  sincos(th, &s, &c);
  J[0][0] = R * c;
  J[0][1] = -r * w * s;
  J[1][0] = R * s;
  J[1][1] = r * w * c;
  H[0][0][0] = 0.0;
  H[0][0][1] = H[0][1][0] = -R * w * s;
  H[0][1][1] = -r * w * w * c;
  H[1][0][0] = 0.0;
  H[1][0][1] = H[1][1][0] = R * w * c;
  H[1][1][1] = -r * w * w * s;
  if (X) *X = r * c;
}

__device__ static void map_jh(int kind, int d, double r0, double r1, const double *xi, Geo3 &g) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      g.J[a][b] = (a == b) ? 1.0 : 0.0;
      for (int c = 0; c < 3; ++c) g.H[a][b][c] = 0.0;
    }
  if (kind == IGA_GEOM_IDENTITY) return;
  double J2[2][2], H2[2][2][2], X;
  ring_jh(r0, r1, xi[0], xi[1], J2, H2, &X);
  if (kind == IGA_GEOM_QUARTER_ANNULUS) {
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        g.J[a][b] = J2[a][b];
        for (int c = 0; c < 2; ++c) g.H[a][b][c] = H2[a][b][c];
      }
    return;
  }
  // revolved ring: rotate (X, Y, 0) about the axis through (-1,-1,-1), direction y
  const double cx = -1.0, cz = -1.0, w = 0.5 * M_PI, phi = w * xi[2];
  double s, c;
  sincos(phi, &s, &c);
  const double a = X - cx, b = 0.0 - cz;
  for (int q = 0; q < 2; ++q) {
    g.J[0][q] = c * J2[0][q];
    g.J[1][q] = J2[1][q];
    g.J[2][q] = -s * J2[0][q];
    for (int q2 = 0; q2 < 2; ++q2) {
      g.H[0][q][q2] = c * H2[0][q][q2];
      g.H[1][q][q2] = H2[1][q][q2];
      g.H[2][q][q2] = -s * H2[0][q][q2];
    }
    g.H[0][q][2] = g.H[0][2][q] = -w * s * J2[0][q];
    g.H[2][q][2] = g.H[2][2][q] = -w * c * J2[0][q];
  }
  g.J[0][2] = w * (-a * s + b * c);
  g.J[1][2] = 0.0;
  g.J[2][2] = w * (-a * c - b * s);
  g.H[0][2][2] = w * w * (-a * c - b * s);
  g.H[1][2][2] = 0.0;
  g.H[2][2][2] = w * w * (a * s - b * c);
}

// inverse of the d x d leading block of J (d = 2 or 3)
__device__ static void inv_small(int d, const double J[3][3], double Ji[3][3]) {
  if (d == 2) {
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    Ji[0][0] = J[1][1] / det;
    Ji[0][1] = -J[0][1] / det;
    Ji[1][0] = -J[1][0] / det;
    Ji[1][1] = J[0][0] / det;
    return;
  }
  const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
  Ji[0][0] = c00 / det;
  Ji[1][0] = c01 / det;
  Ji[2][0] = c02 / det;
  Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
}

// fields[f * ldf + i]: q_aa = -G^{aa}, q_ab = -2 G^{ab} (a < b), q_c = -L_c, ordered
// as in field_desc(): 2D (11, 22, 12, 1, 2), 3D (11, 22, 33, 12, 13, 23, 1, 2, 3).
__global__ void geometry_fields_kernel(int d, int kind, double r0, double r1, double w0,
                                       double w1, double w2, const double *tau1,
                                       const double *tau2, const double *tau3, int n1, int n2,
                                       int n3, double *fields, long long ldf) {
  const long long N = (long long)n1 * n2 * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int i1 = (int)(i % n1);
    const int i2 = (int)((i / n1) % n2);
    const int i3 = (int)(i / ((long long)n1 * n2));
    double xi[3] = {tau1[i1], tau2[i2], d == 3 ? tau3[i3] : 0.0};
    Geo3 g;
    map_jh(kind, d, r0, r1, xi, g);
    double Ji[3][3];
    inv_small(d, g.J, Ji);
    double G[3][3];
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += Ji[a][k] * Ji[b][k];
        G[a][b] = s;
      }
    double lapF[3];
    for (int k = 0; k < d; ++k) {
      double s = 0.0;
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) s += G[a][b] * g.H[k][a][b];
      lapF[k] = s;
    }
    // first-order coefficients: -L_c of -Lap, plus (J^{-1} w)_c of the convective term
    // w . grad_x u = sum_c (J^{-1} w)_c d_c u_hat (Sec. 3.2, constant wind)
    const double wv[3] = {w0, w1, w2};
    double L[3];
    for (int c = 0; c < d; ++c) {
      double s = 0.0, sw = 0.0;
      for (int k = 0; k < d; ++k) {
        s += Ji[c][k] * lapF[k];
        sw += Ji[c][k] * wv[k];
      }
      L[c] = -s - sw;  // the fields hold -L_c
    }
    if (d == 2) {
      fields[0 * ldf + i] = -G[0][0];
      fields[1 * ldf + i] = -G[1][1];
      fields[2 * ldf + i] = -2.0 * G[0][1];
      fields[3 * ldf + i] = -L[0];
      fields[4 * ldf + i] = -L[1];
    } else {
      fields[0 * ldf + i] = -G[0][0];
      fields[1 * ldf + i] = -G[1][1];
      fields[2 * ldf + i] = -G[2][2];
      fields[3 * ldf + i] = -2.0 * G[0][1];
      fields[4 * ldf + i] = -2.0 * G[0][2];
      fields[5 * ldf + i] = -2.0 * G[1][2];
      fields[6 * ldf + i] = -L[0];
      fields[7 * ldf + i] = -L[1];
      fields[8 * ldf + i] = -L[2];
    }
  }
}

void launch_geometry_fields(int d, const iga_geometry &g, const double *tau1, const double *tau2,
                            const double *tau3, int n1, int n2, int n3, double *fields,
                            long long ldf, cudaStream_t s) {
  const long long N = (long long)n1 * n2 * n3;
  const int threads = 256;
  const int blocks = (int)std::min<long long>((N + threads - 1) / threads, 152LL * 16);
  geometry_fields_kernel<<<blocks, threads, 0, s>>>(d, g.kind, g.r_inner, g.r_outer, g.wind[0],
                                                    g.wind[1], d == 3 ? g.wind[2] : 0.0, tau1,
                                                    tau2, tau3, n1, n2, n3, fields, ldf);
  IGA_LAUNCH_CHECK();
}

// Weighted-quadrature Galerkin coefficients (eq. Q with K = I): Q = det(J) J^{-1} J^{-T} at
// the tensor grid of quadrature points x1 x x2 (x x3), and |det J| for the load vector.
__global__ void wq_fields_kernel(int d, int kind, double r0, double r1, const double *x1,
                                 const double *x2, const double *x3, int n1, int n2, int n3,
                                 double *fields, long long ldf) {
  const long long N = (long long)n1 * n2 * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const int i1 = (int)(i % n1);
    const int i2 = (int)((i / n1) % n2);
    const int i3 = (int)(i / ((long long)n1 * n2));
    double xi[3] = {x1[i1], x2[i2], d == 3 ? x3[i3] : 0.0};
    Geo3 g;
    map_jh(kind, d, r0, r1, xi, g);
    double Ji[3][3];
    inv_small(d, g.J, Ji);
    double det;
    if (d == 2) {
      det = g.J[0][0] * g.J[1][1] - g.J[0][1] * g.J[1][0];
    } else {
      det = g.J[0][0] * (g.J[1][1] * g.J[2][2] - g.J[1][2] * g.J[2][1]) -
            g.J[0][1] * (g.J[1][0] * g.J[2][2] - g.J[1][2] * g.J[2][0]) +
            g.J[0][2] * (g.J[1][0] * g.J[2][1] - g.J[1][1] * g.J[2][0]);
    }
    double Q[3][3];
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += Ji[a][k] * Ji[b][k];
        Q[a][b] = det * s;
      }
    if (d == 2) {
      fields[0 * ldf + i] = Q[0][0];
      fields[1 * ldf + i] = Q[1][1];
      fields[2 * ldf + i] = Q[0][1];
      fields[3 * ldf + i] = fabs(det);
    } else {
      fields[0 * ldf + i] = Q[0][0];
      fields[1 * ldf + i] = Q[1][1];
      fields[2 * ldf + i] = Q[2][2];
      fields[3 * ldf + i] = Q[0][1];
      fields[4 * ldf + i] = Q[0][2];
      fields[5 * ldf + i] = Q[1][2];
      fields[6 * ldf + i] = fabs(det);
    }
  }
}

void launch_wq_fields(int d, const iga_geometry &g, const double *x1, const double *x2,
                      const double *x3, int n1, int n2, int n3, double *fields, long long ldf,
                      cudaStream_t s) {
  const long long N = (long long)n1 * n2 * n3;
  const int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 16);
  wq_fields_kernel<<<blocks, 256, 0, s>>>(d, g.kind, g.r_inner, g.r_outer, x1, x2, x3, n1, n2,
                                          n3, fields, ldf);
  IGA_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ band passes
template <class T> __device__ __forceinline__ double ld_val(const T *p) { return (double)__ldg(p); }
// FP32 inputs (the precision form's vectors) are widened on the integer units (fp_widen.h)
template <> __device__ __forceinline__ double ld_val<float>(const float *p) {
  return widen_f32(__ldg(p));
}

// out[o][i] = sum_t band_{order[o]}[c * W + t] * in[i + (start[c] + t - c) * stride],
// c = coordinate of i along dir.  One thread per output point; 32-bit indices
// (N < 2^31): c = (i / divA) mod divB by multiply-shift division, divA = 1, n1 or n1 n2.
// NOUT (1..3) is a template argument: a predicated-off FP64 FMA still takes an issue
// slot on GB300's narrow FP64 unit, so no output's FMAs are issued when it does not exist.
template <class Tin, int W, int NOUT>
__global__ void __launch_bounds__(256) band_pass_kernel(IdxPtr<const Tin> inp, double *out0,
                                                        double *out1, double *out2, int ord0,
                                                        int ord1, int ord2, int dir,
                                                        unsigned N, int stride, FastDiv divA,
                                                        FastDiv divB, BandDev b) {
  pdl_entry();
  const Tin *in = inp.get();
  auto band = [&](int o) { return o == 0 ? b.band0 : (o == 1 ? b.band1 : b.band2); };
  const double *B0 = band(ord0), *B1 = band(ord1), *B2 = band(ord2);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const unsigned qa = dir == 0 ? i : fdiv(i, divA);
    const int c = (int)(qa - fdiv(qa, divB) * divB.d);
    const int st = __ldg(b.start + c);
    const Tin *src = in + (int)i + (st - c) * stride;
    double v[W];
#pragma unroll
    for (int t = 0; t < W; ++t) v[t] = ld_val(src + t * stride);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll
    for (int t = 0; t < W; ++t) a0 = fma(__ldg(B0 + c * W + t), v[t], a0);
    out0[i] = a0;
    if constexpr (NOUT > 1) {
#pragma unroll
      for (int t = 0; t < W; ++t) a1 = fma(__ldg(B1 + c * W + t), v[t], a1);
      out1[i] = a1;
    }
    if constexpr (NOUT > 2) {
#pragma unroll
      for (int t = 0; t < W; ++t) a2 = fma(__ldg(B2 + c * W + t), v[t], a2);
      out2[i] = a2;
    }
  }
}

static int grid_for(long long N, int threads) {
  return (int)std::min<long long>((N + threads - 1) / threads, 152LL * 16);
}

template <class Tin>
void launch_band_pass(IdxPtr<const Tin> in, double *const *outs, const int *orders, int nout,
                      int dir, int n1, int n2, int n3, const BandDev &b, cudaStream_t s,
                      int nrhs) {
  const long long N = (long long)n1 * n2 * n3 * nrhs;
  if (N > kMaxIndex32) throw Error{IGA_ERR_INVALID_ARG, "more than 2^31 - 1 values per operator pass"};
  if (nout < 1 || nout > 3) throw Error{IGA_ERR_INVALID_ARG, "band pass: 1..3 outputs"};
  const int threads = 256, blocks = grid_for(N, threads);
  double *o0 = outs[0], *o1 = nout > 1 ? outs[1] : nullptr, *o2 = nout > 2 ? outs[2] : nullptr;
  const int r0 = orders[0], r1 = nout > 1 ? orders[1] : 0, r2 = nout > 2 ? orders[2] : 0;
  const int stride = dir == 0 ? 1 : (dir == 1 ? n1 : n1 * n2);
  // c = (i / divA) mod divB: dir 0: i mod n1; dir 1: (i / n1) mod n2; dir 2: (i / n1 n2) mod n3
  const FastDiv divA = make_fastdiv(dir == 2 ? (unsigned)(n1 * n2) : (unsigned)n1);
  const FastDiv divB = make_fastdiv(dir == 0 ? (unsigned)n1 : (dir == 1 ? (unsigned)n2 : (unsigned)n3));
#define IGA_BAND_LAUNCH(WW, NO)                                                                \
  launch_pdl(kPdlOperator, band_pass_kernel<Tin, WW, NO>, dim3(blocks), dim3(threads), 0, s, in, \
             o0, o1, o2, r0, r1, r2, dir, (unsigned)N, stride, divA, divB, b)
#define IGA_BAND_CASE(WW)                                     \
  case WW:                                                    \
    if (nout == 1) IGA_BAND_LAUNCH(WW, 1);                    \
    else if (nout == 2) IGA_BAND_LAUNCH(WW, 2);               \
    else IGA_BAND_LAUNCH(WW, 3);                              \
    break;
  switch (b.W) {
    IGA_BAND_CASE(3)
    IGA_BAND_CASE(4)
    IGA_BAND_CASE(5)
    IGA_BAND_CASE(6)
    IGA_BAND_CASE(7)
    default:
      throw Error{IGA_ERR_INVALID_ARG, "band width out of range"};
  }
#undef IGA_BAND_CASE
#undef IGA_BAND_LAUNCH
  IGA_LAUNCH_CHECK();
}

struct BandMulti {
  const double *in[3];
  double *out[6];
  int in_of[6];
  int ord[6];
  int nin, nout;
};

// The band passes of several inputs along one direction in one launch (see
// band_pass_kernel): per point, each input's W taps are loaded once and feed all outputs
// that read it.
template <int W>
__global__ void __launch_bounds__(256) band_pass_multi_kernel(BandMulti m, int dir, unsigned N,
                                                              int stride, FastDiv divA,
                                                              FastDiv divB, BandDev b) {
  pdl_entry();
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const unsigned qa = dir == 0 ? i : fdiv(i, divA);
    const int c = (int)(qa - fdiv(qa, divB) * divB.d);
    const int off = (int)i + (__ldg(b.start + c) - c) * stride;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= m.nin) break;
      const double *src = m.in[a] + off;
      double v[W];
#pragma unroll
      for (int t = 0; t < W; ++t) v[t] = __ldg(src + t * stride);
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        if (q >= m.nout || m.in_of[q] != a) continue;
        const int o = m.ord[q];
        const double *B = (o == 0 ? b.band0 : (o == 1 ? b.band1 : b.band2)) + c * W;
        double acc = 0.0;
#pragma unroll
        for (int t = 0; t < W; ++t) acc = fma(__ldg(B + t), v[t], acc);
        m.out[q][i] = acc;
      }
    }
  }
}

void launch_band_pass_multi(const double *const *ins, int nin, double *const *outs,
                            const int *in_of, const int *orders, int nout, int dir, int n1, int n2,
                            int n3, const BandDev &b, cudaStream_t s, int nrhs) {
  if (nin < 1 || nin > 3 || nout < 1 || nout > 6)
    throw Error{IGA_ERR_INVALID_ARG, "band pass: 1..3 inputs and 1..6 outputs"};
  const long long N = (long long)n1 * n2 * n3 * nrhs;
  if (N > kMaxIndex32) throw Error{IGA_ERR_INVALID_ARG, "more than 2^31 - 1 values per operator pass"};
  BandMulti m{};
  for (int a = 0; a < nin; ++a) m.in[a] = ins[a];
  for (int q = 0; q < nout; ++q) {
    if (in_of[q] < 0 || in_of[q] >= nin) throw Error{IGA_ERR_INVALID_ARG, "band pass input index"};
    m.out[q] = outs[q];
    m.in_of[q] = in_of[q];
    m.ord[q] = orders[q];
  }
  m.nin = nin;
  m.nout = nout;
  const int threads = 256, blocks = grid_for(N, threads);
  const int stride = dir == 0 ? 1 : (dir == 1 ? n1 : n1 * n2);
  const FastDiv divA = make_fastdiv(dir == 2 ? (unsigned)(n1 * n2) : (unsigned)n1);
  const FastDiv divB = make_fastdiv(dir == 0 ? (unsigned)n1 : (dir == 1 ? (unsigned)n2 : (unsigned)n3));
#define IGA_BANDM_CASE(WW)                                                                       \
  case WW:                                                                                       \
    launch_pdl(kPdlOperator, band_pass_multi_kernel<WW>, dim3(blocks), dim3(threads), 0, s, m,   \
               dir, (unsigned)N, stride, divA, divB, b);                                         \
    break;
  switch (b.W) {
    IGA_BANDM_CASE(3)
    IGA_BANDM_CASE(4)
    IGA_BANDM_CASE(5)
    IGA_BANDM_CASE(6)
    IGA_BANDM_CASE(7)
    default:
      throw Error{IGA_ERR_INVALID_ARG, "band width out of range"};
  }
#undef IGA_BANDM_CASE
  IGA_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ contraction pass
// Per-term arguments, resolved on the host: term t reads src[t] (an intermediate of the
// earlier passes) with the band of order[t] along direction 0 and the field coef[t].  The
// kernel unrolls over the terms so that it indexes its parameters statically (no local
// copy of the arrays).
template <class Tin, int W>
__global__ void __launch_bounds__(256) contract_pass_kernel(ContractArgsT<Tin> a, double *out,
                                                            unsigned N, FastDiv div1,
                                                            FastDiv divN1, BandDev b) {
  pdl_entry();
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int c = (int)(i - fdiv(i, div1) * div1.d);         // coordinate along direction 0
    const unsigned ic = i - fdiv(i, divN1) * divN1.d;         // point index of one rhs
    out[i] = contract_point<Tin, W>(a, i, ic, c, b);
  }
}

template <class Tin>
ContractArgsT<Tin> make_contract_args(IdxPtr<const Tin> const *ins, const ContractTerm *terms,
                                      int nterm) {
  if (nterm < 0 || nterm > kMaxFields) throw Error{IGA_ERR_INVALID_ARG, "contraction terms"};
  ContractArgsT<Tin> a{};
  for (int t = 0; t < nterm; ++t) {
    const IdxPtr<const Tin> &in = ins[terms[t].input];
    if (in.idx) throw Error{IGA_ERR_INVALID_ARG, "contraction inputs must be plain pointers"};
    a.src[t] = in.base;
    a.order[t] = terms[t].order;
    a.coef[t] = terms[t].coef;
  }
  a.nterm = nterm;
  return a;
}
template ContractArgsT<double> make_contract_args<double>(IdxPtr<const double> const *,
                                                          const ContractTerm *, int);

template <class Tin>
void launch_contract_pass(IdxPtr<const Tin> const *ins, const ContractTerm *terms, int nterm,
                          double *out, int n1, int n2, int n3, const BandDev &b, cudaStream_t s,
                          int nrhs) {
  const ContractArgsT<Tin> a = make_contract_args<Tin>(ins, terms, nterm);
  const long long N = (long long)n1 * n2 * n3 * nrhs;
  if (N > kMaxIndex32) throw Error{IGA_ERR_INVALID_ARG, "more than 2^31 - 1 values per operator pass"};
  const int threads = 256, blocks = grid_for(N, threads);
  const FastDiv div1 = make_fastdiv((unsigned)n1), divN1 = make_fastdiv((unsigned)(n1 * n2 * n3));
#define IGA_CON_CASE(WW)                                                                   \
  case WW:                                                                                 \
    launch_pdl(kPdlOperator, contract_pass_kernel<Tin, WW>, dim3(blocks), dim3(threads), 0, s, \
               a, out, (unsigned)N, div1, divN1, b);                                           \
    break;
  switch (b.W) {
    IGA_CON_CASE(3)
    IGA_CON_CASE(4)
    IGA_CON_CASE(5)
    IGA_CON_CASE(6)
    IGA_CON_CASE(7)
    default:
      throw Error{IGA_ERR_INVALID_ARG, "band width out of range"};
  }
#undef IGA_CON_CASE
  IGA_LAUNCH_CHECK();
}

template void launch_band_pass<double>(IdxPtr<const double>, double *const *, const int *, int,
                                       int, int, int, int, const BandDev &, cudaStream_t, int);
template void launch_band_pass<float>(IdxPtr<const float>, double *const *, const int *, int, int,
                                      int, int, int, const BandDev &, cudaStream_t, int);
template void launch_contract_pass<double>(IdxPtr<const double> const *, const ContractTerm *, int,
                                           double *, int, int, int, const BandDev &, cudaStream_t,
                                           int);
template void launch_contract_pass<float>(IdxPtr<const float> const *, const ContractTerm *, int,
                                          double *, int, int, int, const BandDev &, cudaStream_t,
                                          int);

// ------------------------------------------------------------------ max |field|
__global__ void field_maxabs_kernel(const double *fields, long long ldf, long long N, int nf,
                                    unsigned long long *out) {
  for (int f = 0; f < nf; ++f) {
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
      m = fmax(m, fabs(fields[f * ldf + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + f, (unsigned long long)__double_as_longlong(m));
  }
}

void launch_field_maxabs(const double *fields, long long ldf, long long N, int nf,
                         unsigned long long *out, cudaStream_t s) {
  IGA_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(unsigned long long) * nf, s));
  field_maxabs_kernel<<<grid_for(N, 256), 256, 0, s>>>(fields, ldf, N, nf, out);
  IGA_LAUNCH_CHECK();
}

template <class Tin, int W> static void preload_op_w() {
  cudaFuncAttributes a;
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, band_pass_kernel<Tin, W, 1>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, band_pass_kernel<Tin, W, 2>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, band_pass_kernel<Tin, W, 3>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, contract_pass_kernel<Tin, W>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, band_pass_multi_kernel<W>));
}

void preload_kernels_geom_op() {
  cudaFuncAttributes a;
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, geometry_fields_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, wq_fields_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, field_maxabs_kernel));
  preload_op_w<double, 3>();
  preload_op_w<double, 4>();
  preload_op_w<double, 5>();
  preload_op_w<double, 6>();
  preload_op_w<double, 7>();
  preload_op_w<float, 3>();
  preload_op_w<float, 4>();
  preload_op_w<float, 5>();
  preload_op_w<float, 6>();
  preload_op_w<float, 7>();
}

}  // namespace iga
