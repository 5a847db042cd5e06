// FP64 mode products of the FD solve (eq. FD2D / FD3D), as GEMMs with layout
// rotation.  A tensor X with scalar index i = i_1 + n_1 (i_2 + n_2 i_3) is read as
// the row-major matrix A[r][k] = X[k + n_1 r] (r = (i_2, i_3), k = i_1); the mode-1
// product with W^T writes out[r + M c] = sum_k A[r][k] W[k][c].  The output's
// fastest index is therefore (i_2, i_3) and the next mode product again contracts
// the contiguous index.  After d products the original order is restored.
// Several right-hand sides stacked as the slowest index stay slowest: with
// P = rows per right-hand side, row = rl + P r writes out[rl + P (c + n r)].
// The diagonal solve of (sum_l I (x) D_l (x) I) is fused into the epilogue of the
// d-th forward product.
#include "iga_internal.h"

namespace iga {

constexpr int kTM = 32, kTN = 64, kKC = 32, kThreads = 256;

template <class Tout>
__global__ void __launch_bounds__(kThreads)
    gemm_fp64_kernel(IdxPtr<const double> Ap, const double *__restrict__ Bt, IdxPtr<Tout> Op,
                     int M, int N, int K, int rows_per, FdScale sc, int has_scale) {
  __shared__ double As[kTM][kKC + 1];
  __shared__ double Bs[kTN][kKC + 1];
  const double *__restrict__ A = Ap.get();
  Tout *__restrict__ O = Op.get();
  const int row0 = blockIdx.x * kTM, col0 = blockIdx.y * kTN;
  const int tm = min(kTM, M - row0), tn = min(kTN, N - col0);
  const int tid = threadIdx.x;
  // work items: 4 consecutive rows x 1 column; rows fastest across threads
  constexpr int kRG = kTM / 4;
  const int nitems = kRG * tn;
  double acc[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.0;
  for (int k0 = 0; k0 < K; k0 += kKC) {
    const int kc = min(kKC, K - k0);
    for (int e = tid; e < kTM * kKC; e += kThreads) {
      const int r = e / kKC, k = e % kKC;
      As[r][k] = (r < tm && k < kc) ? A[(long long)(row0 + r) * K + k0 + k] : 0.0;
    }
    for (int e = tid; e < kTN * kKC; e += kThreads) {
      const int c = e / kKC, k = e % kKC;
      Bs[c][k] = (c < tn && k < kc) ? __ldg(Bt + (long long)(col0 + c) * K + k0 + k) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int it = tid + j * kThreads;
      if (it < nitems) {
        const int rg = it % kRG, c = it / kRG;
        for (int k = 0; k < kc; ++k) {
          const double b = Bs[c][k];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[j][q] = fma(As[4 * rg + q][k], b, acc[j][q]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int it = tid + j * kThreads;
    if (it < nitems) {
      const int rg = it % kRG, c = it / kRG;
      const int col = col0 + c;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = row0 + 4 * rg + q;
        if (4 * rg + q < tm) {
          const int rl = row % rows_per, rr = row / rows_per;
          double v = acc[j][q];
          if (has_scale) {
            double den = sc.lam_r0[rl % sc.n0] + sc.lam_c[col];
            if (sc.lam_r1) den += sc.lam_r1[rl / sc.n0];
            v = v / den;
          }
          O[rl + (long long)rows_per * (col + (long long)N * rr)] = (Tout)v;
        }
      }
    }
  }
}

template <class Tout>
void launch_gemm_fp64(IdxPtr<const double> A, const double *Bt, IdxPtr<Tout> out, int M, int N,
                      int K, const FdScale *scale, cudaStream_t s, int nrhs) {
  dim3 grid((M + kTM - 1) / kTM, (N + kTN - 1) / kTN);
  FdScale sc = scale ? *scale : FdScale{nullptr, nullptr, nullptr, 1};
  gemm_fp64_kernel<Tout><<<grid, kThreads, 0, s>>>(A, Bt, out, M, N, K, M / nrhs, sc,
                                                   scale ? 1 : 0);
  IGA_LAUNCH_CHECK();
}

template void launch_gemm_fp64<double>(IdxPtr<const double>, const double *, IdxPtr<double>, int,
                                       int, int, const FdScale *, cudaStream_t, int);
template void launch_gemm_fp64<float>(IdxPtr<const double>, const double *, IdxPtr<float>, int,
                                      int, int, const FdScale *, cudaStream_t, int);

void preload_kernels_fd64() {
  cudaFuncAttributes a;
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, gemm_fp64_kernel<double>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, gemm_fp64_kernel<float>));
}

}  // namespace iga
