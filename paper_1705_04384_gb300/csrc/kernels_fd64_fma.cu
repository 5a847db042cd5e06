// Folded FP64 mode products of the FD solve (eq. FD2D / FD3D) on FP64 FMAs (CUDA cores).
//
// The same products as fd_fold_mma_kernel (kernels_fd64.cu) -- the folded forward and
// inverse products of a reflection-symmetric pencil, with the same layout rotation and the
// fused diagonal -- on the FMA path instead of mma.sync.  On GB300 the FP64 unit retires
// FMAs about 13 % faster than FP64 MMAs (1243 against 1098 GFLOP/s, fp64_peak.cu).
//
// Output columns are the work unit.  Columns are numbered row-tile-major (row tile of 32
// rows, then the block: even / odd for the forward product, pairs / middle index for the
// inverse one), each costs the FMAs of its contraction, and every warp of a grid sized to
// the SM count takes an equal-cost contiguous range of them (two warps per SM sub-partition,
// the adjacent shares of one sub-partition's warps).  Each block's columns are split into
// runs of balanced length (at most kFmaRun; the same split in every row tile, so that the
// warps of an SM run few distinct loop bodies: with many, the forward product stalled on
// instruction fetch), and a warp covers its range run by run, cutting only the runs at its
// range's ends.  In a run lane l owns row
// 32 rt + l, keeps one accumulator per column of the run, and for each k loads its (folded)
// input entry -- each lane streams its own row through L1 -- and the run's factor entries,
// the same for every lane (broadcast loads of the transposed factor: one base pointer,
// consecutive addresses).  The column count of a run is a template argument: an FP64
// instruction with a false predicate would still take the FP64 unit's issue slot.  Rows
// past M read row 0 and store nothing, so that the loops carry no FP64 masking.
//   forward (DIR 0), even block c < ne:  y_c = sum_{f < h} BfT[f][c] (x_f + x_{n-1-f})
//                                              (+ BfT[h][c] x_h, n odd)
//                    odd block ne + c:   y_{ne+c} = sum_{a < no} BfT[ne+a][ne+c] (x_a - x_{n-1-a})
//   inverse (DIR 1), pair a < h:  pe = sum_{k < ne} BiT[k][a] y_k,  po = sum_{k < no}
//                    BiT[ne+k][a] y_{ne+k};  z_a = pe + po,  z_{n-1-a} = pe - po;
//                    middle index h (n odd):  z_h = sum_{k < ne} BiT[k][h] y_k.
// BfT and BiT are the transposes of the folded factors of kernels_fd64.cu (n x n and
// n x ne).  Each output is written by one lane in a fixed order: bitwise reproducible.
#include "iga_internal.h"

#include <algorithm>
#include <cstdlib>
#include <cstring>

namespace iga {

constexpr int kFmaRows = 32, kFmaWarps = 8, kFmaRun = 32, kFmaPairRun = 16;

struct FmaGeom {
  int n, ne, h;
  int cols0, cols1;  // columns of block 0 / 1 in a row tile (pairs and middle for DIR 1)
  int k0, k1;        // FMAs per lane of a block-0 / block-1 column
  int run_max;       // columns per run
};

// the first column whose cost prefix reaches `target` (columns numbered row-tile-major)
__device__ __forceinline__ long long fma_col_at(const FmaGeom &G, long long target) {
  const long long ct = (long long)G.cols0 * G.k0 + (long long)G.cols1 * G.k1;
  const long long rt = target / ct;
  const long long r = target - rt * ct;
  const long long b0 = (long long)G.cols0 * G.k0;
  long long c;
  if (r <= b0) c = (r + G.k0 - 1) / G.k0;
  else c = G.cols0 + (r - b0 + G.k1 - 1) / G.k1;
  return rt * (G.cols0 + G.cols1) + c;
}

__device__ __forceinline__ void fma_store(double *__restrict__ O, int row, int rows_per, int n,
                                          int col, double v, const double *__restrict__ dinv) {
  const int rl = row % rows_per, rr = row / rows_per;
  if (dinv) v *= __ldg(dinv + rl + (long long)rows_per * col);
  O[rl + (long long)rows_per * (col + (long long)n * rr)] = v;
}

// forward, one parity block: sgn = +1 (even block, K = h folded entries and the middle
// entry when n is odd) or -1 (odd block, K = no); acc[q] gets column col0 + q.  The fold
// x_k + sgn x_{n-1-k} is one FP64 FMA, exactly the sum or the difference.
template <int C>
__device__ __forceinline__ void fwd_block_run(const double *__restrict__ x,
                                              const double *__restrict__ b, int n, int K,
                                              double sgn, bool middle, int h, double (&acc)[C]) {
#pragma unroll 2
  for (int k = 0; k < K; ++k) {
    const double a = fma(sgn, x[n - 1 - k], x[k]);
#pragma unroll
    for (int q = 0; q < C; ++q) acc[q] = fma(a, __ldg(b + (long long)k * n + q), acc[q]);
  }
  if (middle) {  // the middle entry of the even block (n odd)
    const double a = x[h];
#pragma unroll
    for (int q = 0; q < C; ++q) acc[q] = fma(a, __ldg(b + (long long)h * n + q), acc[q]);
  }
}

template <int C>
__device__ __forceinline__ void fwd_run(const double *__restrict__ A,
                                        const double *__restrict__ BT, double *__restrict__ O,
                                        int M, const FmaGeom &G, int rt, int blk, int c0,
                                        int rows_per, const double *__restrict__ dinv) {
  const int row = rt * kFmaRows + (threadIdx.x & 31);
  const bool rv = row < M;
  const double *__restrict__ x = A + (long long)(rv ? row : 0) * G.n;
  double acc[C];
#pragma unroll
  for (int q = 0; q < C; ++q) acc[q] = 0.0;
  const int col0 = (blk ? G.ne : 0) + c0;
  // even block: rows f < h of BfT (and h); odd block: rows ne + a of BfT
  fwd_block_run<C>(x, BT + (blk ? (long long)G.ne * G.n : 0) + col0, G.n, blk ? G.n - G.ne : G.h,
                   blk ? -1.0 : 1.0, !blk && G.ne > G.h, G.h, acc);
  if (rv) {
#pragma unroll
    for (int q = 0; q < C; ++q) fma_store(O, row, rows_per, G.n, col0 + q, acc[q], dinv);
  }
}

// inverse: pairs c0 .. c0 + C - 1 (block 0) or the middle index (block 1, C = 1)
template <int C>
__device__ __forceinline__ void inv_run(const double *__restrict__ A,
                                        const double *__restrict__ BT, double *__restrict__ O,
                                        int M, const FmaGeom &G, int rt, int blk, int c0,
                                        int rows_per) {
  const int row = rt * kFmaRows + (threadIdx.x & 31);
  const bool rv = row < M;
  const int n = G.n, ne = G.ne, no = n - ne;
  const double *__restrict__ x = A + (long long)(rv ? row : 0) * n;
  if (blk) {
    double pe = 0.0;
    const double *__restrict__ b = BT + G.h;
#pragma unroll 4
    for (int k = 0; k < ne; ++k) pe = fma(x[k], __ldg(b + (long long)k * ne), pe);
    if (rv) fma_store(O, row, rows_per, n, G.h, pe, nullptr);
    return;
  }
  double pe[C], po[C];
#pragma unroll
  for (int q = 0; q < C; ++q) pe[q] = po[q] = 0.0;
  const double *__restrict__ b = BT + c0;
#pragma unroll 2
  for (int k = 0; k < ne; ++k) {
    const double a = x[k];
#pragma unroll
    for (int q = 0; q < C; ++q) pe[q] = fma(a, __ldg(b + (long long)k * ne + q), pe[q]);
  }
  b += (long long)ne * ne;
  x += ne;
#pragma unroll 2
  for (int k = 0; k < no; ++k) {
    const double a = x[k];
#pragma unroll
    for (int q = 0; q < C; ++q) po[q] = fma(a, __ldg(b + (long long)k * ne + q), po[q]);
  }
  if (rv) {
#pragma unroll
    for (int q = 0; q < C; ++q) {
      fma_store(O, row, rows_per, n, c0 + q, pe[q] + po[q], nullptr);
      fma_store(O, row, rows_per, n, n - 1 - c0 - q, pe[q] - po[q], nullptr);
    }
  }
}

#define IGA_C8(F, b) F(b + 1) F(b + 2) F(b + 3) F(b + 4) F(b + 5) F(b + 6) F(b + 7) F(b + 8)

template <int DIR>
__device__ __forceinline__ void fma_run_any(int C, const double *A, const double *BT, double *O,
                                            int M, const FmaGeom &G, int rt, int blk, int c0,
                                            int rows_per, const double *dinv) {
  if constexpr (DIR == 0) {
#define IGA_FWD(CC) \
  case CC: fwd_run<CC>(A, BT, O, M, G, rt, blk, c0, rows_per, dinv); break;
    switch (C) {
      IGA_C8(IGA_FWD, 0) IGA_C8(IGA_FWD, 8) IGA_C8(IGA_FWD, 16) IGA_C8(IGA_FWD, 24)
      default: break;
    }
#undef IGA_FWD
  } else {
#define IGA_INV(CC) \
  case CC: inv_run<CC>(A, BT, O, M, G, rt, blk, c0, rows_per); break;
    switch (C) {
      IGA_C8(IGA_INV, 0) IGA_C8(IGA_INV, 8)
      default: break;
    }
#undef IGA_INV
  }
}
#undef IGA_C8

// Virtual warp v = (SM sub-partition slot) * wps + (warp of that slot), as in
// fd_fold_mma_kernel, so that every sub-partition receives the same FP64 work.
template <int DIR>
__global__ void __launch_bounds__(kFmaWarps * 32, 1)
    fd_fold_fma_kernel(IdxPtr<const double> Ap, const double *__restrict__ BT, IdxPtr<double> Op,
                       int M, FmaGeom G, long long nrt, int rows_per, const double *dinv) {
  const int wpb = blockDim.x >> 5, wi = threadIdx.x >> 5, wps = wpb / 4;
  const long long W = (long long)gridDim.x * wpb;
  const long long v = ((long long)blockIdx.x * 4 + wi % 4) * wps + wi / 4;
  const long long total = ((long long)G.cols0 * G.k0 + (long long)G.cols1 * G.k1) * nrt;
  long long it = fma_col_at(G, total * v / W);
  const long long iend = fma_col_at(G, total * (v + 1) / W);
  const int cpt = G.cols0 + G.cols1;
  // programmatic dependent launch, as fd_fold_mma_kernel: wait for the previous product,
  // then let the next one be scheduled
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  const double *__restrict__ A = Ap.get();
  double *__restrict__ O = Op.get();
  while (it < iend) {  // warp-uniform
    const int rt = (int)(it / cpt);
    int c = (int)(it - (long long)rt * cpt);
    const int blk = c >= G.cols0 ? 1 : 0;
    if (blk) c -= G.cols0;
    // the block's columns are split into nr runs of balanced length (at most run_max); the
    // piece of the run that holds c and lies in this warp's range
    const int cols = blk ? G.cols1 : G.cols0;
    const int rmax = (DIR == 1 && blk) ? 1 : G.run_max;
    const int nr = (cols + rmax - 1) / rmax;
    const int r = ((c + 1) * nr + cols - 1) / cols - 1;
    const int run_end = (int)((long long)cols * (r + 1) / nr);
    const int len = (int)min((long long)(run_end - c), iend - it);
    fma_run_any<DIR>(len, A, BT, O, M, G, rt, blk, c, rows_per, dinv);
    it += len;
  }
}

static int num_sms_fma() {
  static int sms[64] = {};
  int dev = 0;
  IGA_CUDA_TRY(cudaGetDevice(&dev));
  int nsm = (dev >= 0 && dev < 64) ? sms[dev] : 0;
  if (nsm == 0) {
    IGA_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (dev >= 0 && dev < 64) sms[dev] = nsm;
  }
  return nsm;
}

void launch_gemm_fp64_fold_fma(int dir, IdxPtr<const double> A, const double *BT,
                               IdxPtr<double> out, int M, int n, int ne, const double *dinv,
                               cudaStream_t s, int nrhs) {
  if (dir != 0 && dir != 1) throw Error{IGA_ERR_INVALID_ARG, "fold_fma: direction 0 or 1"};
  FmaGeom G{};
  G.n = n;
  G.ne = ne;
  G.h = n / 2;
  if (dir == 0) {
    G.cols0 = ne;
    G.cols1 = n - ne;
    G.k0 = ne;
    G.k1 = n - ne;
    G.run_max = kFmaRun;
  } else {
    G.cols0 = n / 2;  // pairs
    G.cols1 = n % 2;  // the middle index
    G.k0 = n;
    G.k1 = ne;
    G.run_max = kFmaPairRun;
  }
  static const int run_cap = [] {
    const char *e = std::getenv("IGA_FMA_RUN");
    const int v = e ? std::atoi(e) : 0;
    return v >= 1 && v <= kFmaRun ? v : kFmaRun;
  }();
  G.run_max = std::min(G.run_max, run_cap);
  const long long nrt = (M + kFmaRows - 1) / kFmaRows;
  const dim3 grid(num_sms_fma()), block(kFmaWarps * 32);
  if (dir == 0)
    launch_pdl(kPdlFd64, fd_fold_fma_kernel<0>, grid, block, 0, s, A, BT, out, M, G, nrt,
               M / nrhs, dinv);
  else
    launch_pdl(kPdlFd64, fd_fold_fma_kernel<1>, grid, block, 0, s, A, BT, out, M, G, nrt,
               M / nrhs, (const double *)nullptr);
  IGA_LAUNCH_CHECK();
}

// Measured on GB300 (FD applies, CUDA events): the FMA kernel is faster when every warp gets
// a few full runs -- 3D n = 130: 1.60 against 1.74 ms per apply, n = 132: 1.65 against 1.89,
// 2D n = 1025: 4.05 against 4.32 -- and slower at 3D n = 65 (165 against 139 us), where a warp
// gets about 7 columns.  So it runs when the columns per warp reach 16.
bool use_fold_fma(long long M, int n) {
  static const int forced = [] {
    const char *e = std::getenv("IGA_FD64");
    if (e && std::strcmp(e, "fma") == 0) return 1;
    if (e && std::strcmp(e, "mma") == 0) return 0;
    return -1;
  }();
  if (forced >= 0) return forced == 1;
  const long long cols = (M + kFmaRows - 1) / kFmaRows * (long long)n;
  return cols >= 16LL * kFmaWarps * num_sms_fma();
}

void preload_kernels_fd64_fma() {
  cudaFuncAttributes a;
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, fd_fold_fma_kernel<0>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, fd_fold_fma_kernel<1>));
}

}  // namespace iga
