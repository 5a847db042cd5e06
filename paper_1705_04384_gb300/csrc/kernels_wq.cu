// Matrix-free weighted-quadrature Galerkin operator (Sec. 2.3, eq. WQapprox) by sum
// factorization:
//   A_wq u = sum_{a,b} (W_d^{(a_d,b_d)} (x) .. (x) W_1^{(a_1,b_1)}) diag(Q_ab(x_q))
//                      (B_d^{(b_d)} (x) .. (x) B_1^{(b_1)}) u,
// a_l = [l == a], b_l = [l == b], Q = det(J) J^{-1} J^{-T} (eq. Q).  Every factor is a
// banded rectangular matrix acting along one direction: the trial functions' values or
// derivatives at the quadrature points (nq x n, expansion onto the quadrature grid) or
// a univariate weighted-quadrature rule (n x nq, contraction back to the test
// functions).  One launch applies several such banded products along one direction:
// term t reads input in[t], applies the band rows of the output coordinate, optionally
// multiplies the input by a pointwise factor first (the Q_ab field on the quadrature
// grid, for the load vector's first contraction), and adds into output out_of[t]; the terms of
// one output are consecutive, so each output is one running sum (a per-output accumulator
// array indexed by a runtime output number compiled to predicated FP64 adds for every slot,
// which take FP64 issue slots even when predicated off).  The operator's last expansion
// pass fans out instead: each derivative of u on the quadrature grid is summed once and
// written once per Q_ab that multiplies it (Q on the output grid), so the contraction
// taps are plain FMAs (multiplying Q in at every contraction tap cost ~WW n / nq times the
// multiplies).
#include "fp_widen.h"
#include "iga_internal.h"

namespace iga {

template <class Tin> __device__ __forceinline__ double wq_ld(const Tin *p) {
  return (double)__ldg(p);
}
// FP32 inputs are widened on the integer units (fp_widen.h)
template <> __device__ __forceinline__ double wq_ld<float>(const float *p) {
  return widen_f32(__ldg(p));
}

// sum_u band[u] src[u L] over the term's band width: WD > 0 the width as a template
// argument (every term of a pass has the same width), fully unrolled; WD = 0 any width.
template <int WD, class Tin>
__device__ __forceinline__ double band_dot(const double *__restrict__ bd, const Tin *src,
                                           unsigned L, int w) {
  double s = 0.0;
  if constexpr (WD > 0) {
#pragma unroll
    for (int u = 0; u < WD; ++u) s = fma(__ldg(bd + u), wq_ld(src + (long long)u * L), s);
  } else {
#pragma unroll 4
    for (int u = 0; u < w; ++u) s = fma(__ldg(bd + u), wq_ld(src + (long long)u * L), s);
  }
  return s;
}
template <int WD, class Tin>
__device__ __forceinline__ double band_dot_coef(const double *__restrict__ bd, const Tin *src,
                                                const double *__restrict__ cf, unsigned L,
                                                int w) {
  double s = 0.0;
  if constexpr (WD > 0) {
#pragma unroll
    for (int u = 0; u < WD; ++u)
      s = fma(__ldg(bd + u), wq_ld(src + (long long)u * L) * __ldg(cf + (long long)u * L), s);
  } else {
#pragma unroll 4
    for (int u = 0; u < w; ++u)
      s = fma(__ldg(bd + u), wq_ld(src + (long long)u * L) * __ldg(cf + (long long)u * L), s);
  }
  return s;
}

// Output point o of one right-hand side = low + L (c + Dout high): low indexes the
// directions faster than the pass, c the pass direction, high the slower ones; the
// input rows of c are start[c] .. start[c] + width - 1 along the pass direction.
template <class Tin, int WD>
__global__ void __launch_bounds__(256)
    wq_pass_kernel(WqPassArgs<Tin> a, unsigned Nout, unsigned L, unsigned Din, FastDiv divL,
                   FastDiv divD, long long in_per_rhs, long long out_per_rhs) {
  pdl_entry();
  const int r = blockIdx.y;
  const Tin *vin = a.vin.get();
  if (a.fan) {  // expansion with the Q factors applied on the output grid
    for (unsigned o = blockIdx.x * blockDim.x + threadIdx.x; o < Nout;
         o += gridDim.x * blockDim.x) {
      const unsigned rest = fdiv(o, divL), low = o - rest * L;
      const unsigned high = fdiv(rest, divD), c = rest - high * divD.d;
      const long long base = (long long)low + (long long)L * Din * high;
#pragma unroll
      for (int t = 0; t < kWqMaxTerms; ++t) {
        if (t >= a.nterm) break;
        const int st = __ldg(a.start[t] + c), w = WD > 0 ? WD : a.width[t];
        const double *bd = a.band[t] + (long long)c * w;
        const Tin *src = (a.in[t] ? a.in[t] : vin) + r * in_per_rhs + base + (long long)L * st;
        const double s = band_dot<WD>(bd, src, L, w);
#pragma unroll
        for (int k = 0; k < kWqMaxFan; ++k) {
          if (k >= a.nfan[t]) break;
          a.fout[t][k][r * out_per_rhs + o] = __ldg(a.fcoef[t][k] + o) * s;
        }
      }
    }
    return;
  }
  for (unsigned o = blockIdx.x * blockDim.x + threadIdx.x; o < Nout; o += gridDim.x * blockDim.x) {
    const unsigned rest = fdiv(o, divL), low = o - rest * L;
    const unsigned high = fdiv(rest, divD), c = rest - high * divD.d;
    const long long base = (long long)low + (long long)L * Din * high;
    // terms come sorted by output: one running sum, stored when the output changes
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < kWqMaxTerms; ++t) {
      if (t >= a.nterm) break;
      const int st = __ldg(a.start[t] + c), w = WD > 0 ? WD : a.width[t];
      const double *bd = a.band[t] + (long long)c * w;
      const Tin *src = (a.in[t] ? a.in[t] : vin) + r * in_per_rhs + base + (long long)L * st;
      const double *cf = a.coef[t] ? a.coef[t] + base + (long long)L * st : nullptr;
      const double s = cf ? band_dot_coef<WD>(bd, src, cf, L, w) : band_dot<WD>(bd, src, L, w);
      acc += s;
      if (t + 1 == a.nterm || a.out_of[t + 1] != a.out_of[t]) {
        a.out[a.out_of[t]][r * out_per_rhs + o] = acc;
        acc = 0.0;
      }
    }
  }
}

template <class Tin>
void launch_wq_pass(const WqPassArgs<Tin> &a, int dir, const int *ext_in, const int *ext_out,
                    int R, cudaStream_t s) {
  if (a.fan) {
    if (a.nterm < 1 || a.nterm > kWqMaxTerms)
      throw Error{IGA_ERR_INVALID_ARG, "weighted-quadrature pass: bad term count"};
    for (int t = 0; t < a.nterm; ++t)
      if (a.nfan[t] < 1 || a.nfan[t] > kWqMaxFan || a.coef[t])
        throw Error{IGA_ERR_INVALID_ARG, "weighted-quadrature pass: bad fan-out"};
  } else if (a.nterm < 1 || a.nterm > kWqMaxTerms || a.nout < 1 || a.nout > kWqMaxOut) {
    throw Error{IGA_ERR_INVALID_ARG, "weighted-quadrature pass: bad term or output count"};
  }
  // the kernel sums consecutive terms of one output: outputs 0 .. nout-1 in order, each
  // with at least one term
  for (int t = 0; t < a.nterm && !a.fan; ++t)
    if (a.out_of[t] != (t ? a.out_of[t - 1] + (a.out_of[t] != a.out_of[t - 1]) : 0))
      throw Error{IGA_ERR_INVALID_ARG, "weighted-quadrature pass: terms not grouped by output"};
  if (!a.fan && a.out_of[a.nterm - 1] != a.nout - 1)
    throw Error{IGA_ERR_INVALID_ARG, "weighted-quadrature pass: output without a term"};
  long long L = 1, H = 1;
  for (int l = 0; l < dir; ++l) L *= ext_in[l];
  for (int l = dir + 1; l < 3; ++l) H *= ext_in[l];
  const long long Din = ext_in[dir], Dout = ext_out[dir];
  const long long Nout = L * Dout * H, Nin = L * Din * H;
  if (Nout * R > kMaxIndex32 || Nin * R > kMaxIndex32)
    throw Error{IGA_ERR_INVALID_ARG, "more than 2^31 - 1 values per weighted-quadrature pass"};
  for (int t = 1; t < a.nterm; ++t)
    if (a.width[t] != a.width[0])
      throw Error{IGA_ERR_INVALID_ARG, "weighted-quadrature pass: terms of unequal width"};
  const int threads = 256;
  const int blocks = (int)std::min<long long>((Nout + threads - 1) / threads, 152LL * 16);
  const dim3 grid(blocks, R), block(threads);
  const FastDiv divL = make_fastdiv((unsigned)L), divD = make_fastdiv((unsigned)Dout);
  // the basis widths p + 1 and the rule widths of p = 2 .. 6 on at least 10 elements
  // (3p + 2) as template arguments; any other width runs the generic loop
  switch (a.width[0]) {
#define IGA_WQ_W(WW)                                                                        \
  case WW:                                                                                   \
    launch_pdl(kPdlOperator, wq_pass_kernel<Tin, WW>, grid, block, 0, s, a, (unsigned)Nout,   \
               (unsigned)L, (unsigned)Din, divL, divD, Nin, Nout);                            \
    break;
    IGA_WQ_W(3) IGA_WQ_W(4) IGA_WQ_W(5) IGA_WQ_W(6) IGA_WQ_W(7) IGA_WQ_W(8) IGA_WQ_W(11)
    IGA_WQ_W(14) IGA_WQ_W(17) IGA_WQ_W(20)
#undef IGA_WQ_W
    default:
      launch_pdl(kPdlOperator, wq_pass_kernel<Tin, 0>, grid, block, 0, s, a, (unsigned)Nout,
                 (unsigned)L, (unsigned)Din, divL, divD, Nin, Nout);
  }
  IGA_LAUNCH_CHECK();
}

template void launch_wq_pass<double>(const WqPassArgs<double> &, int, const int *, const int *,
                                     int, cudaStream_t);
template void launch_wq_pass<float>(const WqPassArgs<float> &, int, const int *, const int *, int,
                                    cudaStream_t);

void preload_kernels_wq() {
  cudaFuncAttributes at;
#define IGA_WQ_PRE(WW)                                                       \
  IGA_CUDA_TRY(cudaFuncGetAttributes(&at, wq_pass_kernel<double, WW>));       \
  IGA_CUDA_TRY(cudaFuncGetAttributes(&at, wq_pass_kernel<float, WW>));
  IGA_WQ_PRE(0) IGA_WQ_PRE(3) IGA_WQ_PRE(4) IGA_WQ_PRE(5) IGA_WQ_PRE(6) IGA_WQ_PRE(7)
  IGA_WQ_PRE(8) IGA_WQ_PRE(11) IGA_WQ_PRE(14) IGA_WQ_PRE(17) IGA_WQ_PRE(20)
#undef IGA_WQ_PRE
}

}  // namespace iga
