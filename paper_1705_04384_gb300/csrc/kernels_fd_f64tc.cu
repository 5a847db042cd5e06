// FP64 FD (eq. FD2D / FD3D) with the mode products on the BF16 tensor cores, exact to FP64
// accuracy: the FP64 form's preconditioner at tensor-core speed (precision IGA_PREC_FP64_TC).
//
// Each mode product C = A B (A: R n^{d-1} x n activation rows, B: an n x n factor stored
// K-contiguous, as in the other FD paths) is evaluated by error-free splitting into
// integer slices (the scheme of Ozaki, Ogita, Oishi and Rump, "Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication", Numer.
// Algorithms 59, 2012), restated here for BF16 products with FP32 accumulation:
//   * every row i of A gets a power of two 2^{e_i} > max_k |A_ik| and every row j of the
//     stored factor (output column j) a power of two 2^{f_j} > max_k |B_kj|;
//   * |A_ik| 2^{56 - e_i}, truncated to an integer F < 2^56, is written in base 2^7 as eight
//     digits 0..127 (most significant first), which carry the sign of A_ik: A_ik =
//     2^{e_i} sum_s d_s 2^{-7(s+1)} up to |A_ik| 2^{-56}; the same for B with digits d'_t;
//   * a digit is an integer of at most 7 bits, exact in BF16; a product of two digits is
//     below 2^14, and a sum of K <= kF64TcMaxK = 148 of them below 2^21.2, exact in FP32.
//     The pairs (s, t) with s + t = w accumulate into one FP32 accumulator G_w (w = 0..7),
//     at most w + 1 pairs: |G_w| <= (w + 1) K 127^2, below 2^24 for every w <= 6 at
//     K <= 148 (and for w = 7 at K <= 130), so G_0..G_6 are the exact integers; only G_7,
//     whose unit is 2^-63 of the result's scale, can round, by at most one unit.  Beyond
//     K = 148 a rounded G_6 (and for larger K G_5, G_4 ...) would cost 2^-56 (2^-49, 2^-42
//     ...) of the scale, more than an FP64 dot product's rounding: the form stops there;
//   * C_ij = 2^{e_i + f_j - 63} sum_{w <= 7} G_w 2^{7 (7 - w)}, rounded once to FP64: two
//     exact 64-bit partial sums and one FMA (recombine).
// The pairs with s + t > 7 are dropped (s + t = 8: 7 pairs of at most K 2^{-56} 2^{e_i + f_j}
// each, the rest 2^-7 smaller) and the digit tails are below 2^-56 of each scale; with the
// final rounding of a result of up to K 2^{e_i + f_j}, the error of C_ij is below about
// 13 K 2^{-56} 2^{e_i + f_j} (2.3e-14 of 2^{e_i + f_j} at K = 130), the size of an FP64 dot
// product's worst-case rounding; measured on random data, 9e-16.
// FP64 arithmetic is limited to three operations per output in the recombination and the FD
// diagonal's multiplication: GB300's FP64 unit is shared by FMAs and the FP64 tensor path,
// and the FP64 FD products run at its ceiling.
//
// Kernels: f64tc_split_kernel (one warp per row of A: the row's scale, then its 8 BF16 digit
// slices; integer operations only) and f64tc_gemm_kernel (one 128-row x n_tile tile per CTA:
// the factor's 8 slices stay in shared memory, the activation's slices stream through a
// TMA ring, one thread issues the 36 slice-pair MMAs per 16-wide K-step into 8 TMEM
// accumulators, eight warps form the FP64 outputs in the layout-rotating order of the other
// FD paths).  Every wait is bounded and reports through the context's device error word.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "context.h"
#include "tc_ptx.cuh"

namespace iga {

constexpr int kSlices = 8;        // base-2^7 digits per value
constexpr int kDigitBits = 7;
constexpr int kF64TcM = 128;      // rows per tile
constexpr int kF64TcThreads = 256;  // 8 epilogue warps: two per TMEM lane quarter
constexpr int kF64TcMaxK = 148;   // the contraction length that keeps G_0..G_6 exact
constexpr int kF64TcSmemBudget = 225 * 1024;  // ring + resident factor (plus 1024 alignment)
constexpr uint32_t kF64TcABytes = kF64TcM * 128;  // one 64-wide K-chunk of one slice

// ------------------------------------------------------------------ splitting
// The BF16 bits of a digit d in [-127, 127]: 2^23 + 128 + d is exact in FP32 (its low byte
// is d + 128), and subtracting 2^23 + 128 leaves d exactly; d has at most 7 significant
// bits, so the upper half of the FP32 word is d in BF16.
__device__ __forceinline__ unsigned short digit_bf16(int d) {
  const float f = __int_as_float(0x4B000000 | (d + 128)) - 8388736.0f;
  return (unsigned short)(__float_as_uint(f) >> 16);
}

// The 56-bit truncated magnitude |x| 2^{56 - e} (x < 2^e in magnitude), from the bits of x.
__device__ __forceinline__ unsigned long long fixed56(unsigned long long bits, int e) {
  const int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long m = bits & ((1ull << 52) - 1);
  int eeff = ex;
  if (ex) m |= 1ull << 52; else eeff = 1;  // subnormal: no hidden bit, exponent of 1
  const int sh = eeff - e - 1019;          // |x| = m 2^{eeff - 1075}; at most 3
  if (sh >= 0) return m << sh;
  return -sh >= 64 ? 0ull : m >> (-sh);
}

// One warp per row of length n of the FP64 input (row r at in + r n): the row's exponent e
// (max |x| < 2^e) to rowexp[r] and the digits of every value to slices[s * sstride + r * kp
// + k].  The padding columns k >= n are never read (the tensor maps end at n).
__global__ void __launch_bounds__(256) f64tc_split_kernel(IdxPtr<const double> inp, int rows, int n,
                                                          int kp, unsigned short *slices,
                                                          long long sstride, int *rowexp) {
  pdl_entry();
  const double *in = inp.get();
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (long long r = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); r < rows;
       r += (long long)gridDim.x * wpb) {
    const unsigned long long *x = (const unsigned long long *)(in + r * n);
    // the largest magnitude: non-negative doubles order as their bit patterns
    unsigned long long mx = 0;
    for (int k = lane; k < n; k += 32) mx = max(mx, x[k] & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int emax = (int)(mx >> 52);
    const int e = emax ? emax - 1022 : -1022;  // max < 2^e (zero and subnormal rows: -1022)
    if (lane == 0) rowexp[r] = e;
    // two adjacent values per lane: one 4-byte store (two BF16 digits) per slice; the row
    // pitch kp is a multiple of 8 values, so pairs starting at even k are 4-byte aligned
    unsigned int *o[kSlices];
#pragma unroll
    for (int s = 0; s < kSlices; ++s) o[s] = (unsigned int *)(slices + s * sstride + r * kp);
    for (int k = 2 * lane; k < n; k += 64) {
      const bool two = k + 1 < n;
      const unsigned long long b0 = x[k], b1 = two ? x[k + 1] : 0ull;
      const unsigned long long F0 = fixed56(b0, e), F1 = fixed56(b1, e);
      const bool n0 = (b0 >> 63) != 0, n1 = (b1 >> 63) != 0;
      // digits 0..3 are bits 55..28 of F, digits 4..7 bits 27..0: two 28-bit halves, so
      // that the digit extraction runs on 32-bit shifts
      const unsigned int h0 = (unsigned int)(F0 >> 28), l0 = (unsigned int)(F0 & 0xFFFFFFFull);
      const unsigned int h1 = (unsigned int)(F1 >> 28), l1 = (unsigned int)(F1 & 0xFFFFFFFull);
#pragma unroll
      for (int s = 0; s < kSlices; ++s) {
        const int sh = kDigitBits * (3 - (s & 3));
        const int d0 = (int)(((s < 4 ? h0 : l0) >> sh) & 127u);
        const int d1 = (int)(((s < 4 ? h1 : l1) >> sh) & 127u);
        const unsigned int lo16 = digit_bf16(n0 ? -d0 : d0), hi16 = digit_bf16(n1 ? -d1 : d1);
        o[s][k >> 1] = lo16 | (hi16 << 16);  // the digit of k + 1 >= n lands in padding
      }
    }
  }
}

// ------------------------------------------------------------------ recombination
// The integer value of an FP32 word that holds an integer of magnitude below 2^25 (below
// 2^24 except G_7 at K = 131, 132), with integer operations only (the float-to-integer
// conversions with 64-bit results run on the FP64 unit).
__device__ __forceinline__ int exact_int_of_f32(uint32_t u) {
  const int ex = (int)((u >> 23) & 0xFFu) - 127;  // 0..24 for a nonzero integer
  if (ex < 0) return 0;
  const unsigned int m = (u & 0x7FFFFFu) | 0x800000u;
  const int mag = (int)(ex <= 23 ? m >> (23 - ex) : m << (ex - 23));
  return (u >> 31) ? -mag : mag;
}

// x 2^E for a normal FP64 x and an integer E, exactly, by adding E to the exponent field
// (ldexp where the result would leave the normal range, which the FD's values do not).
__device__ __forceinline__ double scale_pow2(double x, int E) {
  if (x == 0.0) return 0.0;
  const long long bits = __double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7FF) + E;
  if (be <= 0 || be >= 2047) return ldexp(x, E);
  return __longlong_as_double(bits + ((long long)E << 52));
}

// 2^E sum_w G_w 2^{7 (7 - w)} for the eight exact accumulator words, rounded once: the sum
// splits into H 2^28 + L with H = sum_{w<4} G_w 2^{7 (3 - w)} (|H| < 2^45) and L the same of
// G_4..G_7 (|L| < 2^47), both exact in int64 and in FP64, and one FMA forms H 2^28 + L with a
// single rounding.  Formed with integer operations only (a 128-bit pair normalised to 53
// bits, the same result bit for bit) the epilogue measured slower: 812 against 755 us per FD
// apply at 3D n = 130, although those three FP64 operations take 5.9 us of FP64 issue per
// 8192-output tile.
__device__ __forceinline__ double recombine(const uint32_t (&g)[kSlices], int E) {
  long long H = 0, L = 0;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    H = (H << kDigitBits) + exact_int_of_f32(g[w]);
    L = (L << kDigitBits) + exact_int_of_f32(g[w + 4]);
  }
  return scale_pow2(fma((double)H, 268435456.0, (double)L), E);
}

// 8 columns of one TMEM lane per thread; the wait is in the same statement, so no use of
// r can be scheduled before the load has completed.
__device__ __forceinline__ void tmem_ld8_wait(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
}

struct F64TcEpi {
  double *out;      // FP64 output base
  const int *oidx;  // optional device step index: out += (*oidx) * ostride
  long long ostride;
  int n, ld_out, nmid;  // the rotation of tc_store_rows: row a + n (m + nmid r) ->
                        // a + ld_out (m + nmid col + nmid N r)
  const double *dinv;   // reciprocal FD diagonal in DOF order (nullptr: none)
  int *err;
};

// ------------------------------------------------------------------ slice-product GEMM
// grid (row tiles, column tiles), 128 threads.  Shared memory (after 1024-byte alignment):
// the factor's slices [t][chunk] (n_tile rows x 128 bytes each), then the ring of the
// activation's slice chunks (128 rows x 128 bytes each); the ring depth is what the dynamic
// shared-memory size leaves.  TMEM: accumulator w at columns w n_tile.
// Measured at 3D n = 130: the MMA-issuing thread spends ~160 cycles per M = 128, K = 16
// instruction whatever N (32 or 64) -- staging the activation's K-steps in TMEM with
// tcgen05.cp, so that an MMA reads only the factor tile from shared memory, measured slower
// (1420 against 1211 us per FD apply) -- so the widest tile that TMEM (kSlices n_tile <= 512)
// and shared memory allow is the fastest: fewer instructions per product (64 columns: 907 us
// at n = 130; a last column tile narrowed to its 2 columns' MMA width, N = 16, measured the
// same).
__global__ void __launch_bounds__(kF64TcThreads, 1)
    f64tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                      const __grid_constant__ CUtensorMap mapB, int M, int N, int K, int n_tile,
                      int tmem_cols, uint32_t idesc, const int *__restrict__ rowexp,
                      const int *__restrict__ colexp, F64TcEpi epi) {
  pdl_entry();
  extern __shared__ uint8_t smem_raw[];
  constexpr int kMaxRing = 8;
  __shared__ __align__(8) uint64_t full_bar[kMaxRing];
  __shared__ __align__(8) uint64_t empty_bar[kMaxRing];
  __shared__ __align__(8) uint64_t b_bar;
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int mma_failed;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kF64TcM, c0 = blockIdx.y * n_tile;
  const int nchunks = (K + 63) / 64;
  const uint32_t b_bytes = (uint32_t)n_tile * 128;
  const uint32_t b_total = (uint32_t)(kSlices * nchunks) * b_bytes;
  const int ring = min(kMaxRing, (int)((dynamic_smem_bytes() - 1024u - b_total) / kF64TcABytes));
  uint8_t *sB = smem;
  uint8_t *sA = smem + b_total;
  const int nsteps = kSlices * nchunks;  // activation slice chunks, slice-major

  if (threadIdx.x == 0) {
    for (int q = 0; q < ring; ++q) {
      mbar_init(&full_bar[q], 1);
      mbar_init(&empty_bar[q], 1);
    }
    mbar_init(&b_bar, 1);
    mbar_init(&done_bar, 1);
    mma_failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_base, (uint32_t)tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // the factor's slices for this column tile, once
    mbar_expect_tx(&b_bar, b_total);
    for (int t = 0; t < kSlices; ++t)
      for (int c = 0; c < nchunks; ++c)
        tma_load_3d(sB + (t * nchunks + c) * b_bytes, &mapB, &b_bar, c * 64, c0, t);
    int issued = 0;
    for (int g = 0; g < nsteps; ++g) {
      const int q = g % ring, use = g / ring;
      if (use > 0 && !mbar_wait(&empty_bar[q], (uint32_t)((use - 1) & 1))) {
        atomicExch(epi.err, 11);
        break;
      }
      mbar_expect_tx(&full_bar[q], kF64TcABytes);
      tma_load_3d(sA + q * kF64TcABytes, &mapA, &full_bar[q], (g % nchunks) * 64, m0, g / nchunks);
      ++issued;
    }
    // no copy may still be landing when the CTA exits
    mbar_wait(&b_bar, 0);
    for (int h = issued > ring ? issued - ring : 0; h < issued; ++h)
      mbar_wait(&full_bar[h % ring], (uint32_t)((h / ring) & 1));
  } else if (warp == 1 && lane == 0) {
    bool ok = mbar_wait(&b_bar, 0);
    if (!ok) {
      atomicExch(epi.err, 12);
      mma_failed = 1;
    }
    for (int g = 0; ok && g < nsteps; ++g) {
      const int q = g % ring, use = g / ring;
      if (!mbar_wait(&full_bar[q], (uint32_t)(use & 1))) {
        atomicExch(epi.err, 13);
        mma_failed = 1;
        break;
      }
      tc_fence_after();
      const int s = g / nchunks, c = g % nchunks;
      const int ksteps = min(4, (K - c * 64 + 15) / 16);
      // descriptors: the address field is the byte address / 16, so the K-step j + 1 (32
      // bytes on) is the descriptor + 2 and a factor tile b_bytes on is + b_bytes / 16 (no
      // carry: shared addresses stay below 2^18).  One thread issues 36 x 9 MMAs per tile at
      // 3D n = 130; with both descriptors rebuilt for every MMA the issue loop, not the
      // tensor pipe, set the pace (907 -> 755 us per FD apply once hoisted; issuing a
      // chunk's four K-steps from one asm statement measured the same).
      const uint64_t ad = sw128_desc(smem_u32(sA + q * kF64TcABytes));
      const uint64_t bd0 = sw128_desc(smem_u32(sB + c * b_bytes));
      const uint64_t bstep = (uint64_t)(nchunks * b_bytes) >> 4;  // next slice t
      const uint32_t first = (s > 0 || c > 0) ? 1u : 0u;  // accumulator s + t starts here
      for (int t = 0; t + s < kSlices; ++t) {
        const uint64_t bd = bd0 + (uint64_t)t * bstep;
        const uint32_t dt = tmem + (uint32_t)((s + t) * n_tile);
        mma_issue<1>(dt, ad, bd, idesc, first);
        if (ksteps > 1) mma_issue<1>(dt, ad + 2, bd + 2, idesc, 1u);
        if (ksteps > 2) mma_issue<1>(dt, ad + 4, bd + 4, idesc, 1u);
        if (ksteps > 3) mma_issue<1>(dt, ad + 6, bd + 6, idesc, 1u);
      }
      mma_commit(&empty_bar[q]);
    }
    // committed on every path: TMEM is released only after every issued MMA has completed
    mma_commit(&done_bar);
  }
  __syncwarp();

  const bool have = __all_sync(0xffffffffu, mbar_wait(&done_bar, 0) ? 1 : 0) != 0;
  if (!have) {
    if (lane == 0) atomicExch(epi.err, 14);
  } else if (!*(volatile int *)&mma_failed) {
    tc_fence_after();
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows) and the column half w / 4
    const int q4 = warp & 3, half = warp >> 2;
    const int row = m0 + q4 * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16);
    long long obase = 0;
    const double *dinv_row = nullptr;
    int erow = 0;
    if (row < M) {
      const int a = row % epi.n, rest = row / epi.n;
      const int m = rest % epi.nmid, rr = rest / epi.nmid;
      obase = (long long)a + (long long)epi.ld_out * (m + (long long)epi.nmid * N * rr);
      if (epi.dinv) dinv_row = epi.dinv + a + (long long)epi.n * m;
      erow = rowexp[row];
    }
    const long long cstride = (long long)epi.ld_out * epi.nmid;
    const long long dstride = (long long)epi.n * epi.nmid;
    double *out = epi.out + (epi.oidx ? (long long)(*epi.oidx) * epi.ostride : 0);
    const int cw = n_tile / 2;  // columns of this warp
    for (int cc = half * cw; cc < (half + 1) * cw; cc += 8) {
      uint32_t v[kSlices][8];
#pragma unroll
      for (int w = 0; w < kSlices; ++w) tmem_ld8_wait(tl + (uint32_t)(w * n_tile + cc), v[w]);
      if (row < M) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int col = c0 + cc + q;
          if (col < N) {
            uint32_t g[kSlices];
#pragma unroll
            for (int w = 0; w < kSlices; ++w) g[w] = v[w][q];
            double x = recombine(g, erow + colexp[col] - 63);
            if (dinv_row) x *= __ldg(dinv_row + dstride * col);
            out[obase + cstride * col] = x;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)tmem_cols);
}

// ------------------------------------------------------------------ host side
struct F64TcFd {
  int d = 0, n = 0, kp = 0, M = 0, R_max = 1, nchunks = 0;
  int n_tile = 32, tmem_cols = 256;
  size_t smem = 0;
  uint32_t idesc = 0;
  DevBuf<unsigned short> slA, slVt, slU;  // digit slices (BF16 bits)
  DevBuf<int> rowexp, eVt, eU;
  DevBuf<double> t0, t1;                  // FP64 intermediates
  DevBuf<int> err;
  CUtensorMap mapA{}, mapVt{}, mapU{};
  const double *dinv = nullptr;
};

// The digits of a factor on the host: row j of the n x n matrix B (row-major) gets the
// exponent f_j (max |B_j.| < 2^{f_j}) and its values' 8 digits, as the split kernel does.
static void split_factor_host(const std::vector<double> &B, int n, int kp,
                              std::vector<unsigned short> &sl, std::vector<int> &ex) {
  sl.assign((size_t)kSlices * n * kp, 0);
  ex.assign(n, 0);
  auto bits_of = [](double v) {
    unsigned long long b;
    std::memcpy(&b, &v, 8);
    return b;
  };
  auto bf16_of_digit = [](int dg) {
    const float f = (float)dg;  // |dg| <= 127: exact, and exact in BF16
    unsigned int u;
    std::memcpy(&u, &f, 4);
    return (unsigned short)(u >> 16);
  };
  for (int j = 0; j < n; ++j) {
    unsigned long long mx = 0;
    for (int k = 0; k < n; ++k) mx = std::max(mx, bits_of(B[(size_t)j * n + k]) & 0x7FFFFFFFFFFFFFFFull);
    const int emax = (int)(mx >> 52);
    const int e = emax ? emax - 1022 : -1022;
    ex[j] = e;
    for (int k = 0; k < n; ++k) {
      const unsigned long long b = bits_of(B[(size_t)j * n + k]);
      const int bx = (int)((b >> 52) & 0x7FF);
      unsigned long long m = b & ((1ull << 52) - 1);
      int eeff = bx;
      if (bx) m |= 1ull << 52; else eeff = 1;
      const int sh = eeff - e - 1019;
      const unsigned long long F = sh >= 0 ? (m << sh) : (-sh >= 64 ? 0ull : m >> (-sh));
      const bool neg = (b >> 63) != 0;
      for (int s = 0; s < kSlices; ++s) {
        const int dg = (int)((F >> (kDigitBits * (kSlices - 1 - s))) & 127ull);
        sl[(size_t)s * n * kp + (size_t)j * kp + k] = bf16_of_digit(neg ? -dg : dg);
      }
    }
  }
}

// 3D map over kSlices stacked row-major BF16 matrices (rows x kp, inner extent n: reads
// past n are zero); box = one 128-byte K-chunk x box_rows of one slice.
static void make_slice_map(CUtensorMap &m, const void *base, long long n, long long rows,
                           long long kp, int box_rows) {
  cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)rows, (cuuint64_t)kSlices};
  cuuint64_t strides[2] = {(cuuint64_t)(kp * 2), (cuuint64_t)(rows * kp * 2)};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = tmap_encoder()(
      &m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw Error{IGA_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
}

bool f64tc_supported(int n) { return n >= 1 && n <= kF64TcMaxK; }

F64TcFd *make_f64tc_fd(int d, int n, const Factor1D &f, cudaStream_t s, int R_max,
                       const double *dinv) {
  if (!f64tc_supported(n))
    throw Error{IGA_ERR_UNSUPPORTED, "the FP64 tensor-core FD takes n <= 148"};
  auto *t = new F64TcFd();
  try {
    t->d = d;
    t->n = n;
    t->kp = (n + 7) / 8 * 8;  // 16-byte row pitch for the tensor maps
    long long M = 1;
    for (int l = 0; l < d - 1; ++l) M *= n;
    t->M = (int)M;
    t->R_max = R_max;
    t->nchunks = (n + 63) / 64;
    t->dinv = dinv;
    // 64-column tiles (TMEM holds the kSlices accumulators exactly) when the factor's
    // slices leave room for a 2-stage ring, else 32
    auto ring_for = [&](int nt) {
      const size_t b = (size_t)kSlices * t->nchunks * nt * 128;
      return b >= (size_t)kF64TcSmemBudget ? 0 : (int)std::min<size_t>(8, (kF64TcSmemBudget - b) / kF64TcABytes);
    };
    t->n_tile = ring_for(64) >= 2 ? 64 : 32;
    t->tmem_cols = kSlices * t->n_tile;  // 512 or 256
    const size_t b_total = (size_t)kSlices * t->nchunks * t->n_tile * 128;
    const int ring = ring_for(t->n_tile);
    if (ring < 2) throw Error{IGA_ERR_UNSUPPORTED, "FP64 tensor-core FD: no room for the ring"};
    t->smem = 1024 + b_total + (size_t)ring * kF64TcABytes;
    // instruction descriptor: D = F32, A = B = BF16, K-major, N >> 3, M >> 4
    t->idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(t->n_tile >> 3) << 17) |
               ((uint32_t)(kF64TcM >> 4) << 24);
    // factors: V^T for the forward products, U for the inverse ones (host buffers kept
    // until the stream synchronisation below)
    std::vector<unsigned short> slv, slu;
    std::vector<int> exv, exu;
    split_factor_host(f.Vt, n, t->kp, slv, exv);
    split_factor_host(f.U, n, t->kp, slu, exu);
    auto put = [&](auto &dst, const auto &h) {
      dst.alloc(h.size());
      IGA_CUDA_TRY(cudaMemcpyAsync(dst.ptr, h.data(), h.size() * sizeof(h[0]),
                                   cudaMemcpyHostToDevice, s));
    };
    put(t->slVt, slv);
    put(t->eVt, exv);
    put(t->slU, slu);
    put(t->eU, exu);
    const long long rows = (long long)R_max * M;
    t->slA.alloc((size_t)kSlices * rows * t->kp);
    IGA_CUDA_TRY(cudaMemsetAsync(t->slA.ptr, 0, (size_t)kSlices * rows * t->kp * 2, s));
    t->rowexp.alloc((size_t)rows);
    t->t0.alloc((size_t)rows * n);
    t->t1.alloc((size_t)rows * n);
    t->err.alloc(1);
    IGA_CUDA_TRY(cudaMemsetAsync(t->err.ptr, 0, sizeof(int), s));
    make_slice_map(t->mapA, t->slA.ptr, n, rows, t->kp, kF64TcM);
    make_slice_map(t->mapVt, t->slVt.ptr, n, n, t->kp, t->n_tile);
    make_slice_map(t->mapU, t->slU.ptr, n, n, t->kp, t->n_tile);
    {
      // one attribute per device, the largest any problem needs (it belongs to the kernel)
      static std::atomic<bool> smem_set[64] = {};
      int dev = 0;
      IGA_CUDA_TRY(cudaGetDevice(&dev));
      const bool done = dev >= 0 && dev < 64 && smem_set[dev].load(std::memory_order_acquire);
      std::unique_lock<DeviceLock> lk(device_mutex(), std::defer_lock);
      if (!done) lk.lock();
      if (!done && dev >= 0 && dev < 64 && !smem_set[dev].load(std::memory_order_relaxed)) {
        IGA_CUDA_TRY(cudaFuncSetAttribute(f64tc_gemm_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          1024 + kF64TcSmemBudget));
        smem_set[dev].store(true, std::memory_order_release);
      }
    }
    IGA_CUDA_TRY(cudaStreamSynchronize(s));
  } catch (...) {
    delete t;
    throw;
  }
  return t;
}

void destroy_f64tc_fd(F64TcFd *t) { delete t; }
int *f64tc_error_word(F64TcFd &t) { return t.err.ptr; }

// The chain: for each of the 2d mode products, split its input (the FD input, then the
// previous product's FP64 output) into digit slices and multiply by the factor's slices;
// the d-th product is scaled by the FD diagonal, the last writes `out`.
void f64tc_fd_apply(F64TcFd &t, IdxPtr<const double> in, IdxPtr<double> out, int R,
                    cudaStream_t s) {
  if (R < 1 || R > t.R_max) throw Error{IGA_ERR_INVALID_ARG, "too many right-hand sides"};
  const int rows = R * t.M;
  const long long sstride = (long long)t.R_max * t.M * t.kp;
  const int split_blocks = (int)std::min<long long>((rows + 7) / 8, 152LL * 8);
  const dim3 grid((rows + kF64TcM - 1) / kF64TcM, (t.n + t.n_tile - 1) / t.n_tile);
  IdxPtr<const double> src = in;
  double *bufs[2] = {t.t0.ptr, t.t1.ptr};
  const int total = 2 * t.d;
  for (int g = 0; g < total; ++g) {
    launch_pdl(kPdlTensorCore, f64tc_split_kernel, dim3(split_blocks), dim3(256), 0, s, src, rows,
               t.n, t.kp, t.slA.ptr, sstride, t.rowexp.ptr);
    IGA_LAUNCH_CHECK();
    const bool fwd = g < t.d, last = g == total - 1;
    F64TcEpi e{};
    if (last) {
      e.out = out.base;
      e.oidx = out.idx;
      e.ostride = out.stride;
      if (out.idx && out.off) throw Error{IGA_ERR_INVALID_ARG, "unsupported output offset"};
    } else {
      e.out = bufs[g & 1];
    }
    e.n = t.n;
    e.ld_out = t.n;
    e.nmid = t.M / t.n;
    e.dinv = g == t.d - 1 ? t.dinv : nullptr;
    e.err = t.err.ptr;
    launch_pdl(kPdlTensorCore, f64tc_gemm_kernel, grid, dim3(kF64TcThreads), t.smem, s, t.mapA,
               fwd ? t.mapVt : t.mapU, rows, t.n, t.n, t.n_tile, t.tmem_cols, t.idesc,
               (const int *)t.rowexp.ptr, (const int *)(fwd ? t.eVt.ptr : t.eU.ptr), e);
    IGA_LAUNCH_CHECK();
    if (!last) src = plain_ptr<const double>(bufs[g & 1]);
  }
}

void preload_kernels_fd_f64tc() {
  cudaFuncAttributes a;
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, f64tc_split_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, f64tc_gemm_kernel));
}

}  // namespace iga
