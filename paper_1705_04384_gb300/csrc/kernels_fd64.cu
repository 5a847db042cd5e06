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
            if (sc.dinv) {
              v *= __ldg(sc.dinv + rl + (long long)rows_per * col);
            } else {
              double den = sc.lam_r0[rl % sc.n0] + sc.lam_c[col];
              if (sc.lam_r1) den += sc.lam_r1[rl / sc.n0];
              v = v / den;
            }
          }
          O[rl + (long long)rows_per * (col + (long long)N * rr)] = (Tout)v;
        }
      }
    }
  }
}

// Folded FP64 mode products.  On uniform knots each eigenvector is even or odd under
// the flip i -> n-1-i, so with the eigen-index ordered [even (ne) | odd (no)], V^T and
// U are block diagonal in the basis (x_a +- x_{n-1-a}):
//   forward (DIR 0):  y_c = sum_{f in block(c)} Bf[c][f] * fold(x)_f,
//                     fold(x)_f = x_f + x_{n-1-f} (f < h), x_h (f = h, n odd),
//                                 x_a - x_{n-1-a} (f = ne + a);
//   inverse (DIR 1):  pe_a = sum_{k < ne} Bi[a][k] y_k,  po_a = sum_{k >= ne} Bi[a][k] y_k,
//                     z_a = pe_a + po_a, z_{n-1-a} = pe_a - po_a (a < h), z_h = pe_h.
// Both need n^2 / 2 FMAs per row instead of n^2 (the 1/sqrt(2) of the basis is folded
// into Bf and Bi at setup).  Column tiles of DIR 0 never straddle the two blocks.
template <class Tout, int DIR>
__global__ void __launch_bounds__(kThreads)
    gemm_fp64_fold_kernel(IdxPtr<const double> Ap, const double *__restrict__ Bt, IdxPtr<Tout> Op,
                          int M, int n, int ne, int tiles_e, int rows_per, FdScale sc,
                          int has_scale) {
  __shared__ double As[kTM][kKC + 1];
  __shared__ double Bs[kTN][kKC + 1];
  const double *__restrict__ A = Ap.get();
  Tout *__restrict__ O = Op.get();
  const int h = n / 2, no = n - ne;
  const int row0 = blockIdx.x * kTM;
  int col0, cend, kbeg, kend;
  if (DIR == 0) {
    const bool even = (int)blockIdx.y < tiles_e;
    col0 = even ? blockIdx.y * kTN : ne + (blockIdx.y - tiles_e) * kTN;
    cend = even ? ne : n;
    kbeg = even ? 0 : ne;
    kend = even ? ne : n;
  } else {
    col0 = blockIdx.y * kTN;  // pair index a
    cend = ne;
    kbeg = 0;
    kend = n;
  }
  const int tm = min(kTM, M - row0), tn = min(kTN, cend - col0);
  const int tid = threadIdx.x;
  constexpr int kRG = kTM / 4;
  const int nitems = kRG * tn;
  double acc[2][4][2];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q][0] = acc[j][q][1] = 0.0;
  for (int k0 = kbeg; k0 < kend; k0 += kKC) {
    const int kc = min(kKC, kend - k0);
    for (int e = tid; e < kTM * kKC; e += kThreads) {
      const int r = e / kKC, kk = e % kKC;
      double v = 0.0;
      if (r < tm && kk < kc) {
        const double *x = A + (long long)(row0 + r) * n;
        const int f = k0 + kk;
        if (DIR == 1) {
          v = x[f];
        } else if (f < h) {
          v = x[f] + x[n - 1 - f];
        } else if (f < ne) {
          v = x[h];
        } else {
          v = x[f - ne] - x[n - 1 - (f - ne)];
        }
      }
      As[r][kk] = v;
    }
    for (int e = tid; e < kTN * kKC; e += kThreads) {
      const int c = e / kKC, kk = e % kKC;
      Bs[c][kk] = (c < tn && kk < kc) ? __ldg(Bt + (long long)(col0 + c) * n + k0 + kk) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int it = tid + j * kThreads;
      if (it < nitems) {
        const int rg = it % kRG, c = it / kRG;
        for (int kk = 0; kk < kc; ++kk) {
          const double b = Bs[c][kk];
          const int half = (DIR == 1 && k0 + kk >= ne) ? 1 : 0;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            acc[j][q][half] = fma(As[4 * rg + q][kk], b, acc[j][q][half]);
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
        if (4 * rg + q >= tm) continue;
        const int row = row0 + 4 * rg + q;
        const int rl = row % rows_per, rr = row / rows_per;
        const long long base = rl + (long long)rows_per * (long long)n * rr;
        if (DIR == 0) {
          double v = acc[j][q][0];
          if (has_scale) v *= __ldg(sc.dinv + rl + (long long)rows_per * col);
          O[base + (long long)rows_per * col] = (Tout)v;
        } else {
          const double pe = acc[j][q][0], po = acc[j][q][1];
          if (col < h) {
            O[base + (long long)rows_per * col] = (Tout)(pe + po);
            O[base + (long long)rows_per * (n - 1 - col)] = (Tout)(pe - po);
          } else {
            O[base + (long long)rows_per * col] = (Tout)pe;  // middle index, n odd
          }
        }
      }
    }
  }
}

template <class Tout>
void launch_gemm_fp64_fold(int dir, IdxPtr<const double> A, const double *Bt, IdxPtr<Tout> out,
                           int M, int n, int ne, const FdScale *scale, cudaStream_t s, int nrhs) {
  const int tiles_e = (ne + kTN - 1) / kTN, tiles_o = (n - ne + kTN - 1) / kTN;
  const dim3 grid((M + kTM - 1) / kTM, dir == 0 ? tiles_e + tiles_o : tiles_e);
  FdScale sc = scale ? *scale : FdScale{nullptr, nullptr, nullptr, 1};
  if (dir == 0)
    gemm_fp64_fold_kernel<Tout, 0><<<grid, kThreads, 0, s>>>(A, Bt, out, M, n, ne, tiles_e,
                                                             M / nrhs, sc, scale ? 1 : 0);
  else
    gemm_fp64_fold_kernel<Tout, 1><<<grid, kThreads, 0, s>>>(A, Bt, out, M, n, ne, tiles_e,
                                                             M / nrhs, sc, 0);
  IGA_LAUNCH_CHECK();
}

template void launch_gemm_fp64_fold<double>(int, IdxPtr<const double>, const double *,
                                            IdxPtr<double>, int, int, int, const FdScale *,
                                            cudaStream_t, int);
template void launch_gemm_fp64_fold<float>(int, IdxPtr<const double>, const double *,
                                           IdxPtr<float>, int, int, int, const FdScale *,
                                           cudaStream_t, int);

__global__ void fd_diag_inverse_kernel(const double *__restrict__ lam, int n, int d,
                                       double *__restrict__ dinv, float *__restrict__ dinv32) {
  const long long N = d == 2 ? (long long)n * n : (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double den = lam[i % n] + lam[(i / n) % n];
    if (d == 3) den += lam[i / ((long long)n * n)];
    const double v = 1.0 / den;
    if (dinv) dinv[i] = v;
    if (dinv32) dinv32[i] = (float)v;
  }
}

void launch_fd_diag_inverse(const double *lam, int n, int d, double *dinv, float *dinv32,
                            cudaStream_t s) {
  const long long N = d == 2 ? (long long)n * n : (long long)n * n * n;
  const int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 8);
  fd_diag_inverse_kernel<<<blocks, 256, 0, s>>>(lam, n, d, dinv, dinv32);
  IGA_LAUNCH_CHECK();
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
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, fd_diag_inverse_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, gemm_fp64_fold_kernel<double, 0>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, gemm_fp64_fold_kernel<double, 1>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, gemm_fp64_fold_kernel<float, 1>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, gemm_fp64_fold_kernel<float, 0>));
}

}  // namespace iga
