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
// Both need n^2 / 2 FMAs per row instead of n^2.  The fold uses plain sums and differences
// and Bf, Bi hold the left halves of the rows of V^T and U as they are, so no 1/sqrt(2)
// normalisation appears anywhere.
//
// The products run on the FP64 tensor path (mma.sync m8n8k4 .f64).  On GB300 it has the
// FP64 rate of the CUDA cores (about 2 FMAs per clock per SM), but one warp instruction
// carries 256 FMAs instead of 32, so the kernel is bound by the FP64 pipe rather than by
// instruction issue and load latency.  The work is a list of items (row tile of 8 rows,
// parity block, group of 8 output columns), ordered row-tile-major, and every warp of a
// grid sized to the SM count takes an equal contiguous range of it: each SM sub-partition
// receives the same number of FMAs whatever M and n are.  A warp forms the folded
// A-fragment of a k-step once and feeds up to kMmaNGB column groups of the same row tile
// and block with it.  FP64 FMAs and MMAs share the FP64 pipe of an SM sub-partition and
// their pipe times add (measured on GB300: 619 cycles per m8n8k4, 81 per warp FMA, and a
// batch of fewer than eight FMAs among a warp's MMAs costs an MMA slot).  So the last
// K mod 4 entries of a contraction (n = 65: the middle entry of the even block) run as
// FMAs on the accumulator fragments, in one batch after the run's MMAs, instead of an MMA
// k-step that would be mostly zero padding.  A block's last group, when it has at most
// kPartFma columns and the contraction is at most kPartFmaMaxK long (n = 65: the 33rd even
// column), also runs on FMAs at the end of the run (fold_partial_fma, the column count a
// template argument); otherwise it is padded to a full MMA group with zero factor entries.
// The work split counts both kinds of work in eighths of an MMA.  Each output is written by
// one lane, in a fixed order: the results are bitwise reproducible.
constexpr int kMmaWarps = 4, kMmaWps = 2, kMmaRows = 8, kMmaNGB = 4, kPartFma = 5,
              kPartFmaMaxK = 128;

__device__ __forceinline__ void dmma_m8n8k4(double &c0, double &c1, double a, double b) {
  asm("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
      : "+d"(c0), "+d"(c1)
      : "d"(a), "d"(b));
}

// A block's last column group when it holds PC <= kPartFma columns (cp0 .. cp0+PC-1), on
// FP64 FMAs: lane (g, t) takes row g and the entries k = t (mod 4) of each contraction, four
// of them per batch (loads first), and two xor-shuffles finish the sums.  PC is a
// template argument so that no FMA is issued for a column that does not exist.
template <class Tout, int DIR, int PC>
__device__ __forceinline__ void fold_partial_fma(const double *__restrict__ x, bool rv, int row,
                                                 const double *__restrict__ Bt,
                                                 Tout *__restrict__ O, int n, int ne, int blk,
                                                 int cp0, int Nb, int rows_per,
                                                 const FdScale &sc, int has_scale) {
  const int t = threadIdx.x & 3;
  const int h = n / 2, no = n - ne;
  const int brow0 = (DIR == 0 && blk) ? ne : 0;
  double acc[2][PC];
#pragma unroll
  for (int c = 0; c < PC; ++c) acc[0][c] = acc[1][c] = 0.0;
#pragma unroll
  for (int u = 0; u < (DIR == 1 ? 2 : 1); ++u) {
    if (DIR == 1 && u == 1 && cp0 >= h) break;  // only the middle index: no odd part
    const int K = DIR == 1 ? (u ? no : ne) : Nb;
    const int kb = DIR == 0 ? (blk ? ne : 0) : (u ? ne : 0);
    for (int k0 = t; k0 < K; k0 += 16) {
      double a[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + 4 * q;
        a[q] = 0.0;
        if (rv && k < K) {
          if (DIR != 0) a[q] = x[kb + k];
          else if (!blk) a[q] = k < h ? x[k] + x[n - 1 - k] : x[h];
          else a[q] = x[k] - x[n - 1 - k];
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + 4 * q;
        if (k < K) {
#pragma unroll
          for (int c = 0; c < PC; ++c)
            if (DIR != 1 || u == 0 || cp0 + c < h)
              acc[u][c] = fma(a[q], __ldg(Bt + (long long)(brow0 + cp0 + c) * n + kb + k),
                              acc[u][c]);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < (DIR == 1 ? 2 : 1); ++u)
#pragma unroll
    for (int c = 0; c < PC; ++c) {
      acc[u][c] += __shfl_xor_sync(0xffffffffu, acc[u][c], 1);
      acc[u][c] += __shfl_xor_sync(0xffffffffu, acc[u][c], 2);
    }
  if (!rv) return;
  const int rl = row % rows_per, rr = row / rows_per;
  const long long base = rl + (long long)rows_per * (long long)n * rr;
#pragma unroll
  for (int c = 0; c < PC; ++c) {
    if ((c & 3) != t) continue;
    const int cl = cp0 + c;
    if (DIR != 1) {
      const int col = brow0 + cl;
      double v = acc[0][c];
      if (has_scale) v *= __ldg(sc.dinv + rl + (long long)rows_per * col);
      O[base + (long long)rows_per * col] = (Tout)v;
    } else if (cl < h) {
      O[base + (long long)rows_per * cl] = (Tout)(acc[0][c] + acc[1][c]);
      O[base + (long long)rows_per * (n - 1 - cl)] = (Tout)(acc[0][c] - acc[1][c]);
    } else {
      O[base + (long long)rows_per * cl] = (Tout)acc[0][c];  // middle index, n odd
    }
  }
}

// One run: column groups cg .. cg+len-1 of block blk for the 8 rows of row tile rt.
// DIR 0 / 1: folded forward / inverse product; DIR 2: dense product (no fold, one block
// of n columns, K = n; the caller passes ne = n), for pencils without parity.
template <class Tout, int DIR>
__device__ __forceinline__ void fold_mma_run(const double *__restrict__ A,
                                             const double *__restrict__ Bt, Tout *__restrict__ O,
                                             int M, int n, int ne, int rt, int blk, int cg,
                                             int len, int Nb, int rows_per, const FdScale &sc,
                                             int has_scale) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int h = n / 2, no = n - ne;
  const int row = rt * kMmaRows + g;
  const bool rv = row < M;
  const double *__restrict__ x = A + (long long)(rv ? row : 0) * n;
  const int c0 = cg * 8;                         // first block-local column of the run
  const int brow0 = (DIR == 0 && blk) ? ne : 0;  // factor row of block-local column 0
  // a run that ends with the block's last group, when that group holds at most kPartFma
  // columns and the contraction is short (its FMA chains are latency bound: 2D n = 513
  // measured 4 % slower on FMAs), computes it on FMAs (fold_partial_fma), the rest on MMAs
  const int gb = (Nb + 7) >> 3, pcl = Nb - 8 * (gb - 1);
  const bool part = cg + len == gb && pcl <= kPartFma && Nb <= kPartFmaMaxK;
  if (part) --len;
  double acc[2][kMmaNGB][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int j = 0; j < kMmaNGB; ++j) acc[u][j][0] = acc[u][j][1] = 0.0;
  // the folded input entry k of contraction u (k < that contraction's length)
  auto a_at = [&](int u, int k) -> double {
    if (!rv) return 0.0;
    if (DIR != 0) return x[(u ? ne : 0) + k];
    if (!blk) return k < h ? x[k] + x[n - 1 - k] : x[h];
    return x[k] - x[n - 1 - k];
  };
#pragma unroll
  for (int u = 0; u < (DIR == 1 ? 2 : 1); ++u) {
    // DIR 0: one contraction of length Nb over the block's folded entries;
    // DIR 1: pe over k < ne (u = 0), po over k >= ne (u = 1); DIR 2: k < n.
    // The MMAs take the whole k-steps; the last K mod 4 entries follow on FMAs.
    const int kb = DIR == 0 ? (blk ? ne : 0) : (u ? ne : 0);
    const int K4 = (DIR == 1 ? (u ? no : ne) : Nb) & ~3;
#pragma unroll 2
    for (int s = 0; s < K4; s += 4) {
      const int k = s + t;
      const double a = a_at(u, k);
#pragma unroll
      for (int j = 0; j < kMmaNGB; ++j) {
        // DIR 1: a group starting at or past h holds only the middle index (n odd),
        // whose odd part vanishes
        if (j < len && (DIR != 1 || u == 0 || c0 + 8 * j < h)) {
          // columns past the block's end (its last group may be partial) multiply zeros
          const int cl = c0 + 8 * j + g;
          const double b = cl < Nb ? __ldg(Bt + (long long)(brow0 + cl) * n + kb + k) : 0.0;
          dmma_m8n8k4(acc[u][j][0], acc[u][j][1], a, b);
        }
      }
    }
  }
  // The last K mod 4 entries of each contraction (n = 65: the middle entry of the even
  // block) on FP64 FMAs into the accumulator fragments (lane (g, t) holds row g, columns
  // 2t and 2t+1), one batch after all of the run's MMAs: 2 FMAs per group and entry in
  // place of an MMA whose k-step would be mostly zero padding.
#pragma unroll
  for (int u = 0; u < (DIR == 1 ? 2 : 1); ++u) {
    const int kb = DIR == 0 ? (blk ? ne : 0) : (u ? ne : 0);
    const int K = DIR == 1 ? (u ? no : ne) : Nb;
    for (int k = K & ~3; k < K; ++k) {
      const double a = a_at(u, k);
#pragma unroll
      for (int j = 0; j < kMmaNGB; ++j) {
        if (j < len && (DIR != 1 || u == 0 || c0 + 8 * j < h)) {
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const int cl = c0 + 8 * j + 2 * t + i;
            const double b = cl < Nb ? __ldg(Bt + (long long)(brow0 + cl) * n + kb + k) : 0.0;
            acc[u][j][i] = fma(a, b, acc[u][j][i]);
          }
        }
      }
    }
  }
  if (part) {
    const int cp0 = 8 * (gb - 1);
    switch (pcl) {
      case 1: fold_partial_fma<Tout, DIR, 1>(x, rv, row, Bt, O, n, ne, blk, cp0, Nb, rows_per, sc, has_scale); break;
      case 2: fold_partial_fma<Tout, DIR, 2>(x, rv, row, Bt, O, n, ne, blk, cp0, Nb, rows_per, sc, has_scale); break;
      case 3: fold_partial_fma<Tout, DIR, 3>(x, rv, row, Bt, O, n, ne, blk, cp0, Nb, rows_per, sc, has_scale); break;
      case 4: fold_partial_fma<Tout, DIR, 4>(x, rv, row, Bt, O, n, ne, blk, cp0, Nb, rows_per, sc, has_scale); break;
      default: fold_partial_fma<Tout, DIR, 5>(x, rv, row, Bt, O, n, ne, blk, cp0, Nb, rows_per, sc, has_scale); break;
    }
  }
  if (!rv) return;
  const int rl = row % rows_per, rr = row / rows_per;
  const long long base = rl + (long long)rows_per * (long long)n * rr;
  // lane (g, t) holds row g, columns 2t and 2t+1 of each 8 x 8 tile
#pragma unroll
  for (int j = 0; j < kMmaNGB; ++j) {
    if (j >= len) continue;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int cl = c0 + 8 * j + 2 * t + i;
      if (cl >= Nb) continue;
      if (DIR != 1) {
        const int col = brow0 + cl;
        double v = acc[0][j][i];
        if (has_scale) v *= __ldg(sc.dinv + rl + (long long)rows_per * col);
        O[base + (long long)rows_per * col] = (Tout)v;
      } else {
        const double pe = acc[0][j][i], po = acc[1][j][i];
        if (cl < h) {
          O[base + (long long)rows_per * cl] = (Tout)(pe + po);
          O[base + (long long)rows_per * (n - 1 - cl)] = (Tout)(pe - po);
        } else {
          O[base + (long long)rows_per * cl] = (Tout)pe;  // middle index, n odd
        }
      }
    }
  }
}

// Cost of a contraction of length K for one column group, in eighths of an MMA (about one
// warp FMA each): an MMA per whole k-step and two FMAs per remaining entry.
__device__ __forceinline__ int contraction_cost(int K) { return 8 * (K >> 2) + 2 * (K & 3); }

// Cost of column group j of a row tile: its contraction(s) (a partial last group is padded
// to a full MMA group) plus, in the forward product, the fold add of each k-step shared by
// a run of up to four groups.
__device__ __forceinline__ int fold_group_cost(int DIR, int j, int n, int ne, int g0) {
  const int no = n - ne;
  const int blk = j >= g0 ? 1 : 0;
  const int Nb = (DIR == 0 && blk) ? no : ne;
  const int jl = blk ? j - g0 : j, gb = (Nb + 7) >> 3, pc = Nb - 8 * (gb - 1);
  if (jl == gb - 1 && pc <= kPartFma && Nb <= kPartFmaMaxK) {
    // fold_partial_fma: per batch of 4 entries, a fold add (forward) and pc FMAs
    auto fcost = [&](int K) { return 4 * ((((K + 3) >> 2) + 3) >> 2); };
    const int h = n / 2, cp0 = 8 * (gb - 1);
    if (DIR != 1) return fcost(Nb) * (pc + (DIR == 0 ? 1 : 0)) + 2 * pc;
    const int pairs = max(0, min(Nb, h) - cp0);
    return fcost(ne) * pc + (pairs ? fcost(no) * pairs : 0) + 2 * pc + 2 * pairs;
  }
  if (DIR == 2) return contraction_cost(Nb);
  if (DIR == 0) return contraction_cost(Nb) + (Nb >> 2) / 2;
  return contraction_cost(ne) + (8 * j < n / 2 ? contraction_cost(no) : 0);
}

// First item of the cost share `target` (0 <= target <= total): the smallest item i with
// prefix cost(i) >= target, items ordered row-tile-major.
__device__ long long fold_item_at(int DIR, long long target, long long C, int gpr, int n, int ne,
                                  int g0) {
  const long long rt = target / C;
  long long r = target - rt * C;
  int j = 0;
  while (r > 0 && j < gpr) r -= fold_group_cost(DIR, j++, n, ne, g0);
  return rt * gpr + j;
}

// Virtual warp v = (SM sub-partition slot) * wps + (warp of that slot): the wps warps that
// share an SM sub-partition take adjacent cost shares, so every sub-partition receives
// the same FP64 work (up to one item) whatever the item costs are.
template <class Tout, int DIR>
__global__ void __launch_bounds__(kMmaWarps * 32 * kMmaWps)
    fd_fold_mma_kernel(IdxPtr<const double> Ap, const double *__restrict__ Bt, IdxPtr<Tout> Op,
                       int M, int n, int ne, int g0, int g1, long long nrt, int rows_per,
                       FdScale sc, int has_scale) {
  // programmatic dependent launch: this grid computes its work split before waiting for
  // the previous product's output, then lets the next product be scheduled (its blocks
  // wait in griddepcontrol.wait until this grid has completed).  Triggering only after
  // the wait keeps at most one product waiting ahead: triggered at entry, back-to-back FD
  // applies let launches cascade and settle unevenly on the SMs (2x slower).
  const int wpb = blockDim.x >> 5, wps = wpb / kMmaWarps, wi = threadIdx.x >> 5;
  const long long W = (long long)gridDim.x * wpb;
  const long long v = ((long long)blockIdx.x * kMmaWarps + wi % kMmaWarps) * wps + wi / kMmaWarps;
  const int gpr = g0 + g1;  // column groups per row tile
  long long C = 0;          // cost of one row tile
  for (int j = 0; j < gpr; ++j) C += fold_group_cost(DIR, j, n, ne, g0);
  const long long total = C * nrt;
  long long it = fold_item_at(DIR, total * v / W, C, gpr, n, ne, g0);
  const long long iend =
      fold_item_at(DIR, total * (v + 1) / W, C, gpr, n, ne, g0);
  const int no = n - ne;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
  const double *__restrict__ A = Ap.get();
  Tout *__restrict__ O = Op.get();
  while (it < iend) {  // warp-uniform
    const int rt = (int)(it / gpr);
    int cg = (int)(it - (long long)rt * gpr);
    const int blk = cg >= g0 ? 1 : 0;
    if (blk) cg -= g0;
    const int Nb = (DIR == 0 && blk) ? no : ne;
    const long long blk_end = (long long)rt * gpr + (blk ? gpr : g0);
    const int len = (int)min((long long)kMmaNGB, min(iend, blk_end) - it);
    fold_mma_run<Tout, DIR>(A, Bt, O, M, n, ne, rt, blk, cg, len, Nb, rows_per, sc, has_scale);
    it += len;
  }
}

static int num_sms() {
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

template <class Tout>
void launch_gemm_fp64_fold(int dir, IdxPtr<const double> A, const double *Bt, IdxPtr<Tout> out,
                           int M, int n, int ne, const FdScale *scale, cudaStream_t s, int nrhs) {
  const int no = n - ne;
  // column groups per row tile: DIR 0 has the even (ne) and odd (no) blocks, DIR 1 the
  // ne pairs (g1 = 0)
  const int g0 = (ne + 7) / 8, g1 = dir == 0 ? (no + 7) / 8 : 0;
  const long long nrt = (M + kMmaRows - 1) / kMmaRows;
  // two warps per SM sub-partition: while one waits on its loads the other keeps the
  // sub-partition's FP64 MMA unit busy
  constexpr int wps = kMmaWps;
  const dim3 grid(num_sms()), block(32 * kMmaWarps * wps);
  FdScale sc = scale ? *scale : FdScale{nullptr, nullptr, nullptr, 1};
  if (dir == 0)
    launch_pdl(kPdlFd64, fd_fold_mma_kernel<Tout, 0>, grid, block, 0, s, A, Bt, out, M, n, ne, g0,
               g1, nrt, M / nrhs, sc, scale ? 1 : 0);
  else
    launch_pdl(kPdlFd64, fd_fold_mma_kernel<Tout, 1>, grid, block, 0, s, A, Bt, out, M, n, ne, g0,
               g1, nrt, M / nrhs, sc, 0);
  IGA_LAUNCH_CHECK();
}

// Dense FP64 mode product on the FP64 tensor path (no parity: wind-shifted pencils):
// out[rl + P (c + n r)] = sum_k A[row][k] Bt[c][k] (times dinv with a scale).
template <class Tout>
void launch_gemm_fp64_dense_mma(IdxPtr<const double> A, const double *Bt, IdxPtr<Tout> out,
                                int M, int n, const FdScale *scale, cudaStream_t s, int nrhs) {
  const int g0 = (n + 7) / 8;
  const long long nrt = (M + kMmaRows - 1) / kMmaRows;
  constexpr int wps = kMmaWps;
  const dim3 grid(num_sms()), block(32 * kMmaWarps * wps);
  FdScale sc = scale ? *scale : FdScale{nullptr, nullptr, nullptr, 1};
  launch_pdl(kPdlFd64, fd_fold_mma_kernel<Tout, 2>, grid, block, 0, s, A, Bt, out, M, n, n, g0, 0,
             nrt, M / nrhs, sc, scale ? 1 : 0);
  IGA_LAUNCH_CHECK();
}

template void launch_gemm_fp64_dense_mma<double>(IdxPtr<const double>, const double *,
                                                 IdxPtr<double>, int, int, const FdScale *,
                                                 cudaStream_t, int);
template void launch_gemm_fp64_dense_mma<float>(IdxPtr<const double>, const double *,
                                                IdxPtr<float>, int, int, const FdScale *,
                                                cudaStream_t, int);

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

__global__ void fd_diag_inverse3_kernel(const double *__restrict__ lam1,
                                        const double *__restrict__ lam2,
                                        const double *__restrict__ lam3, int n, int d,
                                        double *__restrict__ dinv, float *__restrict__ dinv32) {
  const long long N = d == 2 ? (long long)n * n : (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double den = lam1[i % n] + lam2[(i / n) % n];
    if (d == 3) den += lam3[i / ((long long)n * n)];
    const double v = 1.0 / den;
    if (dinv) dinv[i] = v;
    if (dinv32) dinv32[i] = (float)v;
  }
}

void launch_fd_diag_inverse3(const double *lam1, const double *lam2, const double *lam3, int n,
                             int d, double *dinv, float *dinv32, cudaStream_t s) {
  const long long N = d == 2 ? (long long)n * n : (long long)n * n * n;
  const int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 8);
  fd_diag_inverse3_kernel<<<blocks, 256, 0, s>>>(lam1, lam2, lam3, n, d, dinv, dinv32);
  IGA_LAUNCH_CHECK();
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
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, fd_diag_inverse3_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, fd_fold_mma_kernel<double, 0>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, fd_fold_mma_kernel<double, 1>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, fd_fold_mma_kernel<float, 0>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, fd_fold_mma_kernel<float, 1>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, fd_fold_mma_kernel<double, 2>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, fd_fold_mma_kernel<float, 2>));
}

}  // namespace iga
