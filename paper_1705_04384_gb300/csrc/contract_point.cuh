// One output of the operator's final pass (eq. collocation by sum factorization): the
// banded mode product along direction 0 of each input, contracted with the geometry
// coefficient fields at the collocation point.  Shared by contract_pass_kernel and the
// fused contraction + first CGS2 pass of an Arnoldi step, so that both compute w bit for bit
// alike.
#pragma once

#include "fp_widen.h"
#include "iga_internal.h"

namespace iga {

template <class Tin> struct ContractArgsT {
  const Tin *src[kMaxFields];
  int order[kMaxFields];
  const double *coef[kMaxFields];
  int nterm;
};

template <class T> __device__ __forceinline__ double contract_ld(const T *p) {
  return (double)__ldg(p);
}
// FP32 inputs are widened on the integer units (fp_widen.h)
template <> __device__ __forceinline__ double contract_ld<float>(const float *p) {
  return widen_f32(__ldg(p));
}

// i: flattened index over the stacked right-hand sides, ic: the point index of one right-hand
// side, c: its coordinate along direction 0
template <class Tin, int W>
__device__ __forceinline__ double contract_point(const ContractArgsT<Tin> &a, long long i,
                                                 unsigned ic, int c, const BandDev &b) {
  const int st = __ldg(b.start + c);
  const long long base = i + (st - c);
  double acc = 0.0;
#pragma unroll
  for (int t = 0; t < kMaxFields; ++t) {
    if (t >= a.nterm) break;
    const Tin *src = a.src[t] + base;
    const int o = a.order[t];
    const double *B = (o == 0 ? b.band0 : (o == 1 ? b.band1 : b.band2)) + c * W;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < W; ++q) s = fma(__ldg(B + q), contract_ld(src + q), s);
    acc = fma(__ldg(a.coef[t] + ic), s, acc);
  }
  return acc;
}

}  // namespace iga

namespace iga {
// Contraction arguments from the operator's pass plan (inputs must be plain pointers).
template <class Tin>
ContractArgsT<Tin> make_contract_args(IdxPtr<const Tin> const *ins, const ContractTerm *terms,
                                      int nterm);
}  // namespace iga
