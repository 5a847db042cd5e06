// FD solve (eq. FD2D / FD3D) with the mode products on the 5th-generation tensor
// cores (tcgen05): TF32 or BF16 operands, FP32 accumulation in tensor memory.
// Error-compensated TF32 (the TF32X3 precision): every operand x is held as two TF32
// tensors, hi = tf32(x) and lo = tf32(x - hi), and each product accumulates
// A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo * lo term, 2^-22 relative, is dropped): three
// MMAs per K-step on twice the staged bytes, for products close to FP32 accuracy.
//
// Each mode product is the GEMM D[M x N] = A[M x K] * B[K x N] of the layout-rotating
// scheme used by the FP64 path (A: activation rows with the contracted index
// contiguous; B: an n x n factor stored K-contiguous), M = n^{d-1}, N = K = n.
// One CTA computes a 128-row tile:
//   warp 0 / lane 0   TMA producer: 128-byte K-chunks of A and B (128B swizzle) into a
//                     kStages-deep ring, one mbarrier per stage;
//   warp 1 / lane 0   MMA issuer: tcgen05.mma (M = 128, N = n_tile, K = 8 / 16 per
//                     instruction) into a TMEM accumulator; tcgen05.commit frees a
//                     stage and finally signals the epilogue;
//   warps 0..3        epilogue: tcgen05.ld of their 32 TMEM lanes, optional division by
//                     lambda_i + mu_j (+ nu_k) (the FD diagonal), conversion, and stores
//                     in the rotated layout (row index fastest, so stores coalesce).
// Every wait is bounded (about one second); a wait that runs out records an error in
// a device word that the host reads after the solve, and the CTA still releases its
// tensor memory before it exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "context.h"
#include "fp_widen.h"
#include "tc_ptx.cuh"

namespace iga {

constexpr int kTcThreads = 128;
constexpr int kTileM = 128;
constexpr int kStages = 4;
// ------------------------------------------------------------------ GEMM kernel
enum { kOutF32 = 0, kOutBF16 = 1, kOutF64 = 2 };

struct TcEpi {
  void *out;        // output base (element type by kind)
  const int *oidx;  // optional device step index: out += (*oidx) * ostride elements
  long long ostride;
  int kind;         // kOutF32 / kOutBF16 / kOutF64
  int tf32_round;   // round FP32 outputs to TF32 (operands of the next TF32 product)
  float *out_lo;    // split TF32 operands: TF32 rounding of the remainder (nullptr: none)
  int n;            // extent of the fastest component of a row index
  int ld_out;       // stride of that component in the output
  int nmid;         // rows per right-hand side / n  (n^{d-2})
  const float *dinv;  // reciprocal FD diagonal in DOF order (nullptr: no scaling)
  int *err;
};

// Epilogue of one 128 x n_tile tile for the 32 rows (TMEM lanes) of one warp: tcgen05.ld of
// 16 columns at a time, optional FD diagonal, conversion, stores in the rotated layout.
// Row = a + n (m + nmid r) (a: fastest component, m: middle, r: right-hand side); the output
// index a + ld_out (m + nmid col + nmid N r) keeps r slowest.  The diagonal's entries of the
// next 16 columns are loaded before this chunk's stores: loaded next to each store they
// waited behind it, a memory latency per column (a persistent CTA's second product, the one
// with the diagonal, took three times as long as its first).  Called by all 32 lanes (the
// TMEM load is warp-collective).  SPLIT: an FP32 output that feeds the next split-TF32
// product is stored as hi = tf32(x) at out and tf32(x - hi) at out_lo when out_lo is set.
template <bool SPLIT = false>
__device__ __forceinline__ void tc_store_rows(uint32_t tl, int row, int M, int c0, int N,
                                              int n_tile, const TcEpi &epi) {
  long long obase = 0;
  const float *dinv_row = nullptr;  // the FD diagonal in DOF order: a + n (m + nmid col)
  if (row < M) {
    const int a = row % epi.n, rest = row / epi.n;
    const int m = rest % epi.nmid, rr = rest / epi.nmid;
    obase = (long long)a + (long long)epi.ld_out * (m + (long long)epi.nmid * N * rr);
    if (epi.dinv) dinv_row = epi.dinv + a + (long long)epi.n * m;
  }
  const long long cstride = (long long)epi.ld_out * epi.nmid;
  const long long dstride = (long long)epi.n * epi.nmid;
  const long long off = epi.oidx ? (long long)(*epi.oidx) * epi.ostride : 0;
  auto load_dv = [&](int cc, float (&dv)[16]) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int col = c0 + cc + j;
      dv[j] = (dinv_row && col < N) ? __ldg(dinv_row + dstride * col) : 1.0f;
    }
  };
  float dv[16];
  load_dv(0, dv);
  for (int cc = 0; cc < n_tile; cc += 16) {
    float dn[16];
    if (cc + 16 < n_tile) load_dv(cc + 16, dn);
    uint32_t v[16];
    tmem_ld16(tl + (uint32_t)cc, v);
    if (row < M) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = c0 + cc + j;
        if (col < N) {
          float x = __uint_as_float(v[j]);
          if (dinv_row) x *= dv[j];
          const long long o = off + obase + cstride * col;
          if (epi.kind == kOutF32) {
            const float hi = epi.tf32_round ? round_tf32(x) : x;
            ((float *)epi.out)[o] = hi;
            if (SPLIT && epi.out_lo) epi.out_lo[o] = round_tf32(x - hi);
          } else if (epi.kind == kOutBF16) {
            ((__nv_bfloat16 *)epi.out)[o] = __float2bfloat16_rn(x);
          } else {
            ((double *)epi.out)[o] = widen_f32(x);  // on the integer units (fp_widen.h)
          }
        }
      }
    }
    if (cc + 16 < n_tile) {
#pragma unroll
      for (int j = 0; j < 16; ++j) dv[j] = dn[j];
    }
  }
}

// Ring depth of the one-tile kernel: at most min(kStages, K chunks), and for the split TF32
// kind (four tiles per chunk) at most what kSplitRingBytes holds.  The depth is chosen on the
// host -- the autotuner times 2 stages and the most allowed: a deeper ring hides more TMA
// latency, a shallower one lets more CTAs share an SM -- and reaches the kernel through the
// dynamic shared-memory size, of which the ring takes all but the 1024 alignment bytes.  The
// split budget leaves room for the static shared memory within the 227 KB a CTA may have.
constexpr int kSplitRingBytes = 225 * 1024;
__host__ __device__ constexpr int tc_stage_bytes(bool split, int n_tile) {
  return (split ? 2 : 1) * (kTileM * 128 + n_tile * 128);
}
__host__ __device__ constexpr int tc_split_max_stages(int nchunks, int n_tile) {
  const int s = nchunks < kStages ? nchunks : kStages;
  const int fit = kSplitRingBytes / tc_stage_bytes(true, n_tile);
  return s < fit ? s : fit;
}

// mapA2 / mapB2: the lo parts of A and B for KIND 2 (not read by the other kinds).
template <int KIND>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapA2,
                   const __grid_constant__ CUtensorMap mapB2, int M, int N, int K, int n_tile,
                   int tmem_cols, uint32_t idesc, TcEpi epi) {
  pdl_entry();  // before any global access, TMEM allocation included
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t a_bytes = kTileM * 128, b_bytes = (uint32_t)n_tile * 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTileM, c0 = blockIdx.y * n_tile;
  constexpr int kbox = KIND == 1 ? 64 : 32;  // elements per 128-byte row
  constexpr int kmma = KIND == 1 ? 16 : 8;   // K per instruction (32 bytes)
  constexpr bool split = KIND == 2;
  constexpr uint32_t kTiles = split ? 2u : 1u;  // tiles of A (and of B) per stage
  const int nchunks = (K + kbox - 1) / kbox;
  // the ring has min(stages, nchunks) stages: a short contraction (K = n, two or three
  // 128-byte chunks at the usual n) takes less shared memory, so more CTAs share an SM
  const int nstage = min(min(kStages, nchunks),
                         (int)((dynamic_smem_bytes() - 1024u) / (kTiles * (a_bytes + b_bytes))));
  uint8_t *sA = smem;
  uint8_t *sB = smem + nstage * a_bytes;
  // split kind: the lo tiles follow (every tile stays 1024-byte aligned: n_tile % 16 == 0)
  uint8_t *sA2 = sB + nstage * b_bytes;
  uint8_t *sB2 = sA2 + nstage * a_bytes;

  __shared__ int mma_failed;
  if (threadIdx.x == 0) {
    for (int s = 0; s < nstage; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
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
    int issued = 0;
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % nstage, use = c / nstage;
      if (use > 0 && !mbar_wait(&empty_bar[s], (uint32_t)((use - 1) & 1))) {
        atomicExch(epi.err, 1);
        break;
      }
      mbar_expect_tx(&full_bar[s], kTiles * (a_bytes + b_bytes));
      tma_load_2d(sA + s * a_bytes, &mapA, &full_bar[s], c * kbox, m0);
      tma_load_2d(sB + s * b_bytes, &mapB, &full_bar[s], c * kbox, c0);
      if constexpr (split) {
        tma_load_2d(sA2 + s * a_bytes, &mapA2, &full_bar[s], c * kbox, m0);
        tma_load_2d(sB2 + s * b_bytes, &mapB2, &full_bar[s], c * kbox, c0);
      }
      ++issued;
    }
    // no copy may still be landing in shared memory when the CTA exits: wait (bounded)
    // for the last uses of the ring (on the normal path the MMAs consumed them already)
    for (int h = issued > nstage ? issued - nstage : 0; h < issued; ++h)
      mbar_wait(&full_bar[h % nstage], (uint32_t)((h / nstage) & 1));
  } else if (warp == 1 && lane == 0) {
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % nstage, use = c / nstage;
      if (!mbar_wait(&full_bar[s], (uint32_t)(use & 1))) {
        atomicExch(epi.err, 2);
        mma_failed = 1;
        break;
      }
      tc_fence_after();
      const int rem = K - c * kbox;
      const int ksteps = min(kbox / kmma, (rem + kmma - 1) / kmma);
      const uint32_t a0 = smem_u32(sA + s * a_bytes), b0 = smem_u32(sB + s * b_bytes);
      const uint32_t a2 = smem_u32(sA2 + s * a_bytes), b2 = smem_u32(sB2 + s * b_bytes);
      for (int j = 0; j < ksteps; ++j) {
        // the correction terms first, the leading term last (all into one accumulator)
        if constexpr (split) {
          mma_issue<KIND>(tmem, sw128_desc(a0 + 32u * j), sw128_desc(b2 + 32u * j), idesc,
                          (c > 0 || j > 0) ? 1u : 0u);
          mma_issue<KIND>(tmem, sw128_desc(a2 + 32u * j), sw128_desc(b0 + 32u * j), idesc, 1u);
        }
        mma_issue<KIND>(tmem, sw128_desc(a0 + 32u * j), sw128_desc(b0 + 32u * j), idesc,
                        (split || c > 0 || j > 0) ? 1u : 0u);
      }
      mma_commit(&empty_bar[s]);
    }
    // committed on every path: done_bar completes once every MMA issued above has, so
    // tensor memory is never released under an MMA still writing it
    mma_commit(&done_bar);
  }
  __syncwarp();

  // epilogue (all four warps; warp w owns TMEM lanes 32w..32w+31 = rows m0+32w..)
  // warp-uniform so that the .sync.aligned tensor-memory loads stay convergent
  const bool have = __all_sync(0xffffffffu, mbar_wait(&done_bar, 0) ? 1 : 0) != 0;
  if (!have) {
    if (lane == 0) atomicExch(epi.err, 3);
  } else if (*(volatile int *)&mma_failed) {
    // the accumulator is incomplete (the error word is already set): store nothing
  } else {
    tc_fence_after();
    const int row = m0 + warp * 32 + lane;
    tc_store_rows<split>(tmem + ((uint32_t)(warp * 32) << 16), row, M, c0, N, n_tile, epi);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)tmem_cols);
}

// ------------------------------------------------------------------ persistent GEMM kernel
// The same product with a grid of at most (SMs x resident CTAs) that loops over the tiles,
// row tile fastest (the order in which the one-tile grid above is launched).  Per CTA the
// setup (barriers, TMEM allocation, tensor-map fetch) is paid once, the TMA ring runs
// ahead across tile boundaries, and two TMEM accumulators let the epilogue of tile i
// overlap the main loop of tile i + 1.  The one-tile kernel runs its phases in series:
// measured at 2D n = 1025 with 8 right-hand sides, its tensor pipe is busy 27 % of the
// cycles its CTAs are resident, with L2 at 18 % and DRAM at 6 % of their peaks.
//   warp 0 / lane 0   TMA producer over the CTA's (tile, chunk) sequence;
//   warp 1            allocates 2 x tmem_cols TMEM columns; lane 0 issues the MMAs of the
//                     CTA's i-th tile into accumulator i & 1 once the epilogue has drained
//                     it, commits each ring stage back to the producer and the finished
//                     accumulator to the epilogue;
//   warps 2..5        epilogue; warp w may access TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31.
// Selected per shape by the autotuner (see persistent_candidate); checked against the
// oracle on a GB300 with IGA_TC_PERSISTENT=2 (tests/test_gpu_mixed.py), and its barrier
// protocol (ring phases, accumulator hand-over) is simulated on the host in
// tests/test_tc_persistent_protocol.py.
constexpr int kTcpThreads = 192;
constexpr int kTcpMaxStages = 8;
constexpr size_t kTcpRingBytes = 200 * 1024;  // ring budget per CTA (stages x stage bytes)

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int KIND>
__global__ void __launch_bounds__(kTcpThreads, 1)
    tc_gemm_persistent_kernel(const __grid_constant__ CUtensorMap mapA,
                              const __grid_constant__ CUtensorMap mapB, int M, int N, int K,
                              int n_tile, int tmem_cols, uint32_t idesc, int nstage, TcEpi epi) {
  pdl_entry();  // before any global access, TMEM allocation included
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[kTcpMaxStages];
  __shared__ __align__(8) uint64_t empty_bar[kTcpMaxStages];
  __shared__ __align__(8) uint64_t accf_bar[2];  // accumulator b holds a finished tile
  __shared__ __align__(8) uint64_t acce_bar[2];  // accumulator b drained by the epilogue
  __shared__ __align__(8) uint64_t fin_bar;      // every MMA of this CTA has completed
  __shared__ uint32_t tmem_base;
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t a_bytes = kTileM * 128, b_bytes = (uint32_t)n_tile * 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kbox = KIND == 0 ? 32 : 64;  // elements per 128-byte row
  constexpr int kmma = KIND == 0 ? 8 : 16;   // K per instruction (32 bytes)
  const int nchunks = (K + kbox - 1) / kbox;
  const int nmt = (M + kTileM - 1) / kTileM, nnt = (N + n_tile - 1) / n_tile;
  const long long ntiles = (long long)nmt * nnt;
  uint8_t *sA = smem;
  uint8_t *sB = smem + nstage * a_bytes;

  if (threadIdx.x == 0) {
    for (int s = 0; s < nstage; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], 4);  // one arrival per epilogue warp
    }
    mbar_init(&fin_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(&tmem_base, 2u * (uint32_t)tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;  // chunks issued so far (ring slot g % nstage, use g / nstage)
      bool ok = true;
      for (long long tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int m0 = (int)(tile % nmt) * kTileM, c0 = (int)(tile / nmt) * n_tile;
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int s = (int)(g % nstage);
          const long long use = g / nstage;
          if (use > 0 && !mbar_wait(&empty_bar[s], (uint32_t)((use - 1) & 1))) {
            atomicExch(epi.err, 4);
            ok = false;
            break;
          }
          mbar_expect_tx(&full_bar[s], a_bytes + b_bytes);
          tma_load_2d(sA + s * a_bytes, &mapA, &full_bar[s], c * kbox, m0);
          tma_load_2d(sB + s * b_bytes, &mapB, &full_bar[s], c * kbox, c0);
        }
      }
      // no copy may be in flight when the CTA exits: wait (bounded) until the last nstage
      // chunks issued have landed (on the normal path the MMAs have consumed them all)
      for (long long h = g > nstage ? g - nstage : 0; h < g; ++h)
        mbar_wait(&full_bar[h % nstage], (uint32_t)((h / nstage) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long g = 0;
      int i = 0;  // tiles of this CTA so far
      bool ok = true;
      for (long long tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x, ++i) {
        const int b = i & 1, ub = i >> 1;
        if (ub > 0 && !mbar_wait(&acce_bar[b], (uint32_t)((ub - 1) & 1))) {
          atomicExch(epi.err, 5);
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(b * tmem_cols);
        for (int c = 0; c < nchunks; ++c, ++g) {
          const int s = (int)(g % nstage);
          const long long use = g / nstage;
          if (!mbar_wait(&full_bar[s], (uint32_t)(use & 1))) {
            atomicExch(epi.err, 6);
            ok = false;
            break;
          }
          tc_fence_after();
          const int rem = K - c * kbox;
          const int ksteps = min(kbox / kmma, (rem + kmma - 1) / kmma);
          const uint32_t a0 = smem_u32(sA + s * a_bytes), b0 = smem_u32(sB + s * b_bytes);
          for (int j = 0; j < ksteps; ++j)
            mma_issue<KIND>(dt, sw128_desc(a0 + 32u * j), sw128_desc(b0 + 32u * j), idesc,
                            (c > 0 || j > 0) ? 1u : 0u);
          mma_commit(&empty_bar[s]);
        }
        if (ok) mma_commit(&accf_bar[b]);
      }
      // tensor memory is freed only after every MMA issued here has completed
      mma_commit(&fin_bar);
      if (!mbar_wait(&fin_bar, 0)) atomicExch(epi.err, 8);
    }
  } else {
    const int q = warp & 3;  // TMEM lane quarter of this warp
    int i = 0;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
      const int b = i & 1, ub = i >> 1;
      // warp-uniform so that the .sync.aligned tensor-memory loads stay convergent
      const bool have =
          __all_sync(0xffffffffu, mbar_wait(&accf_bar[b], (uint32_t)(ub & 1)) ? 1 : 0) != 0;
      if (!have) {
        if (lane == 0) atomicExch(epi.err, 7);
        break;
      }
      tc_fence_after();
      const int m0 = (int)(tile % nmt) * kTileM, c0 = (int)(tile / nmt) * n_tile;
      tc_store_rows(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * tmem_cols),
                    m0 + q * 32 + lane, M, c0, N, n_tile, epi);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce_bar[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 2u * (uint32_t)tmem_cols);
}

// FP64 vector (unpadded) -> TF32-rounded FP32 / BF16 tensor with padded fastest index.
// out_lo (TF32 only; nullptr: none): tf32((float)x - hi), the split form's lo part.
template <class T>
__global__ void pack_kernel(IdxPtr<const double> inp, T *__restrict__ out, float *__restrict__ out_lo,
                            unsigned N, FastDiv divn, int ld) {
  pdl_entry();
  const double *in = inp.get();
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const unsigned q = fdiv(i, divn);
    const long long o = (long long)(i - q * divn.d) + (long long)ld * q;
    if constexpr (sizeof(T) == 4) {
      const float xf = (float)in[i];
      const float hi = round_tf32(xf);
      out[o] = hi;
      if (out_lo) out_lo[o] = round_tf32(xf - hi);  // xf - hi is exact
    } else {
      out[o] = __float2bfloat16_rn((float)in[i]);
    }
  }
}

// ------------------------------------------------------------------ host side
struct TcFd {
  int d = 0, n = 0, prec = 0, kpad = 0, M = 0;  // M = rows of one right-hand side (n^{d-1})
  int R_max = 1;
  int esize = 4, n_tile = 0, n_ntiles = 0, tmem_cols = 0;
  size_t smem = 0;
  // persistent kernel (tc_gemm_persistent_kernel): ring depth, shared memory, CTAs per SM
  int persistent = 0, p_nstage = 0, p_cps = 0;
  int ring = 0;  // stages of the one-tile kernel's ring
  size_t p_smem = 0;
  uint32_t idesc = 0;
  bool split = false;  // error-compensated TF32: every operand as hi and lo TF32 tensors
  DevBuf<uint8_t> P0, Ta, Tb;
  DevBuf<uint8_t> P0lo, Talo, Tblo;  // split only
  DevBuf<int> err;
  CUtensorMap mapP0{}, mapTa{}, mapTb{}, mapVt{}, mapU{};
  CUtensorMap mapP0lo{}, mapTalo{}, mapTblo{}, mapVtlo{}, mapUlo{};  // split only
  const float *dinv32 = nullptr;
  const void *vt_dev = nullptr, *u_dev = nullptr;
  const void *vt_lo_dev = nullptr, *u_lo_dev = nullptr;  // split only
};

// A GEMM operand: its tensor map and, for the split kind, the map of its lo part.
struct TcOp {
  const CUtensorMap *hi, *lo;
};

static void make_map(CUtensorMap &m, const void *base, int elem_bf16, long long n_inner,
                     long long rows, long long ld, int box_rows);
static void gemm(TcFd &t, TcOp A, TcOp B, const TcEpi &epi, int R, cudaStream_t s);

static int num_sms_tc() {
  int dev = 0, nsm = 0;
  IGA_CUDA_TRY(cudaGetDevice(&dev));
  IGA_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  return nsm;
}

// Column-tile shape of the mode products: N = n_tile output columns per CTA (a
// multiple of 16, <= 256), the factor's TMA box and the instruction descriptor follow.
// persistent: the tile loop of tc_gemm_persistent_kernel, with the deepest ring that fits
// kTcpRingBytes and as many CTAs per SM as shared memory and tensor memory (two
// accumulators of tmem_cols columns each, 512 columns per SM) allow.
// ring: stages of the one-tile kernel's ring (0: the most allowed); not used by the persistent
// kernel, whose ring fills kTcpRingBytes.
static void set_tile(TcFd &t, int n_tile, int persistent = 0, int ring = 0) {
  const bool bf = t.prec == IGA_PREC_BF16;
  if (t.split && persistent) throw Error{IGA_ERR_UNSUPPORTED, "split TF32 runs on the one-tile kernel"};
  t.n_tile = n_tile;
  t.persistent = persistent;
  t.n_ntiles = (t.n + n_tile - 1) / n_tile;
  t.tmem_cols = 32;
  while (t.tmem_cols < n_tile) t.tmem_cols *= 2;
  const int kbox = bf ? 64 : 32, nchunks = (t.n + kbox - 1) / kbox;
  const int most = t.split ? tc_split_max_stages(nchunks, n_tile) : std::min(kStages, nchunks);
  const int nstage = ring > 0 ? std::min(ring, most) : most;
  t.ring = nstage;
  t.smem = 1024 + (size_t)nstage * tc_stage_bytes(t.split, n_tile);
  // instruction descriptor: D = F32; A, B = TF32 (2) or BF16 (1); K-major; N >> 3; M >> 4
  const uint32_t fmt = bf ? 1u : 2u;
  t.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n_tile >> 3) << 17) |
            ((uint32_t)(kTileM >> 4) << 24);
  make_map(t.mapVt, t.vt_dev, bf, t.n, t.n, t.kpad, n_tile);
  make_map(t.mapU, t.u_dev, bf, t.n, t.n, t.kpad, n_tile);
  if (t.split) {
    make_map(t.mapVtlo, t.vt_lo_dev, 0, t.n, t.n, t.kpad, n_tile);
    make_map(t.mapUlo, t.u_lo_dev, 0, t.n, t.n, t.kpad, n_tile);
  }
  if (persistent) {
    const size_t stage = (size_t)kTileM * 128 + (size_t)n_tile * 128;
    t.p_nstage = (int)std::max<size_t>(2, std::min<size_t>(kTcpMaxStages, kTcpRingBytes / stage));
    t.p_smem = 1024 + (size_t)t.p_nstage * stage;
    int cps = 0;
    if (bf)
      IGA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &cps, tc_gemm_persistent_kernel<1>, kTcpThreads, t.p_smem));
    else
      IGA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &cps, tc_gemm_persistent_kernel<0>, kTcpThreads, t.p_smem));
    t.p_cps = std::max(1, std::min(cps, 512 / (2 * t.tmem_cols)));
  }
}

// Which kernels the autotuner times.  Measured on GB300 (2D n = 1025, TF32, fastest tile of
// each): with one right-hand side the one-tile kernel is faster (85.5 against 118.7 us per
// FD apply: 45 tiles leave no second tile per CTA to overlap), with eight the persistent
// kernel is (287 against 311 us).  IGA_TC_PERSISTENT unset: the persistent kernel is a
// candidate for problems set up for at least 4 right-hand sides; 0: never; 1: always;
// 2: the only candidate (to check it against the oracle).
static int persistent_mode() {
  const char *e = std::getenv("IGA_TC_PERSISTENT");
  if (!e || !e[0]) return -1;
  return (e[0] == '1' || e[0] == '2') ? e[0] - '0' : 0;
}
static bool persistent_candidate(const TcFd &t) {
  if (t.split) return false;  // the persistent kernel has no split kind
  const int m = persistent_mode();
  return m > 0 || (m < 0 && t.R_max >= 4);
}

// Autotuner: time the 2d mode products of one FD apply (R_max right-hand sides) for each
// candidate column tile -- the padded width split into the fewest parts of at most 256
// columns and up to 5 more (narrower tiles put more CTAs on the GPU at the cost of
// re-reading the row tile), and 256, 128, 64 for n > 256 -- and keep the fastest; on the
// one-tile kernel each width with a 2-stage ring and with the deepest allowed.  The choice
// is cached per (device, d, n, precision, R_max) so that every problem of one shape runs the
// same kernels.
struct TcTileChoice {
  int n_tile, persistent, ring;
};
static void autotune(TcFd &t, cudaStream_t s) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, int>, TcTileChoice> cache;
  int dev = 0;
  IGA_CUDA_TRY(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, t.d, t.n, t.prec, t.R_max);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      set_tile(t, it->second.n_tile, it->second.persistent, it->second.ring);
      return;
    }
  }
  std::vector<int> widths;
  // IGA_TC_TILE=<multiple of 16, at most 256 and n rounded up to 16>: the only column tile
  // (pins the configuration, e.g. for a profiler run, under which the timings that rank the
  // candidates are distorted)
  const char *tile_env = std::getenv("IGA_TC_TILE");
  const int forced_tile = tile_env ? std::atoi(tile_env) : 0;
  if (forced_tile >= 16 && forced_tile <= 256 && forced_tile % 16 == 0 &&
      forced_tile <= (t.n + 15) / 16 * 16) {
    widths = {forced_tile};
  } else {
    // the padded width split into p0 .. p0 + 5 balanced parts (p0: the fewest parts of at most
    // 256 columns), each rounded up to 16: no nearly empty last tile (n = 1025 in 256-column
    // tiles left a fifth tile of one column, a full MMA width of work), and tile counts that
    // fill whole waves of the persistent grid
    const int p0 = (t.n + 255) / 256;
    for (int parts = p0; parts <= p0 + 5; ++parts) {
      const int nt = ((t.n + parts - 1) / parts + 15) / 16 * 16;
      if (nt <= 256 && std::find(widths.begin(), widths.end(), nt) == widths.end())
        widths.push_back(nt);
    }
    // and, for wide problems, the powers of two (2D n = 1025 with one right-hand side runs
    // fastest in 64-column tiles: 77 against 84 us per FD apply for the best balanced width)
    if (t.n > 256)
      for (int nt : {256, 128, 64})
        if (std::find(widths.begin(), widths.end(), nt) == widths.end()) widths.push_back(nt);
  }
  // IGA_TC_RING=<stages>: the one-tile kernel's only ring depth (with IGA_TC_TILE, pins the
  // whole configuration for a profiler run)
  const char *ring_env = std::getenv("IGA_TC_RING");
  const int forced_ring = ring_env ? std::atoi(ring_env) : 0;
  std::vector<TcTileChoice> cand;
  if (persistent_mode() != 2 || t.split)
    for (int nt : widths) {
      if (forced_ring > 0) {
        cand.push_back({nt, 0, forced_ring});  // set_tile clamps it to what is allowed
        continue;
      }
      cand.push_back({nt, 0, 0});
      const int nchunks = (t.n + (t.prec == IGA_PREC_BF16 ? 63 : 31)) /
                          (t.prec == IGA_PREC_BF16 ? 64 : 32);
      const int most =
          t.split ? tc_split_max_stages(nchunks, nt) : std::min(kStages, nchunks);
      if (most > 2) cand.push_back({nt, 0, 2});
    }
  if (persistent_candidate(t))
    for (int nt : widths) cand.push_back({nt, 1, 0});
  TcTileChoice best = cand[0];
  if (cand.size() > 1) {
    // shared: the candidates are this library's preloaded kernels, launched on this problem's
    // own stream, so the timing runs beside other threads' eigensolves and autotunes (timings
    // stay exposed to whatever else runs on the GPU, as they always were to other solves), but
    // never during a graph capture
    const double tw = wall_seconds();
    std::shared_lock<DeviceLock> dlk(device_mutex());
    const double tl = wall_seconds();
    cudaEvent_t e0, e1;
    IGA_CUDA_TRY(cudaEventCreate(&e0));
    IGA_CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    for (const auto &cd : cand) {
      set_tile(t, cd.n_tile, cd.persistent, cd.ring);
      TcEpi e{};
      e.kind = t.prec == IGA_PREC_BF16 ? kOutBF16 : kOutF32;
      e.tf32_round = t.split ? 1 : 0;
      e.n = t.n;
      e.ld_out = t.kpad;
      e.nmid = t.M / t.n;
      e.err = t.err.ptr;
      auto chain_once = [&]() {
        for (int g = 0; g < 2 * t.d; ++g) {
          e.out = (g & 1) ? t.Tb.ptr : t.Ta.ptr;
          if (t.split) e.out_lo = (float *)((g & 1) ? t.Tblo.ptr : t.Talo.ptr);
          const TcOp A = (g & 1) ? TcOp{&t.mapTa, &t.mapTalo} : TcOp{&t.mapP0, &t.mapP0lo};
          const TcOp B = g < t.d ? TcOp{&t.mapVt, &t.mapVtlo} : TcOp{&t.mapU, &t.mapUlo};
          gemm(t, A, B, e, t.R_max, s);
        }
      };
      chain_once();
      IGA_CUDA_TRY(cudaEventRecord(e0, s));
      for (int rep = 0; rep < 3; ++rep) chain_once();
      IGA_CUDA_TRY(cudaEventRecord(e1, s));
      IGA_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      IGA_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best = cd;
      }
      if (verbose_level() >= 1)
        std::fprintf(stderr,
                     "iga autotune d=%d n=%d prec=%d R=%d n_tile=%d%s ring=%d: %.1f us/apply\n",
                     t.d, t.n, t.prec, t.R_max, cd.n_tile, cd.persistent ? " persistent" : "",
                     cd.persistent ? t.p_nstage : t.ring, 1000.f * ms / 3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    IGA_CUDA_TRY(cudaMemsetAsync(t.err.ptr, 0, sizeof(int), s));
    if (verbose_level() >= 2)
      std::fprintf(stderr, "iga autotune d=%d n=%d R=%d: lock wait %.1f ms, %zu candidates "
                   "timed in %.1f ms\n", t.d, t.n, t.R_max, 1e3 * (tl - tw), cand.size(),
                   1e3 * (wall_seconds() - tl));
  }
  set_tile(t, best.n_tile, best.persistent, best.ring);
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = best;
}

int tc_fd_tile(const TcFd &t) { return t.n_tile; }

// The driver's cuTensorMapEncodeTiled, looked up once (shared with kernels_fd_f64tc.cu).
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
  static std::mutex mu;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    IGA_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                  cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p)
      throw Error{IGA_ERR_CUDA, "cuTensorMapEncodeTiled not available"};
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2D map over a row-major matrix: inner extent n_inner (elements read past it are
// zero), rows, row pitch ld elements; box = one 128-byte row segment x box_rows.
static void make_map(CUtensorMap &m, const void *base, int elem_bf16, long long n_inner,
                     long long rows, long long ld, int box_rows) {
  const int es = elem_bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)n_inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = tmap_encoder()(
      &m, elem_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
      const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    throw Error{IGA_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
}

TcFd *make_tc_fd(int d, int n, int precision, const Factor1D &f, cudaStream_t s, int R_max,
                 const float *dinv32) {
  auto *t = new TcFd();
  try {
    t->d = d;
    t->n = n;
    t->prec = precision;
    const bool bf = precision == IGA_PREC_BF16;
    t->split = precision == IGA_PREC_TF32X3;
    t->esize = bf ? 2 : 4;
    t->kpad = f.kpad;
    long long M = 1;
    for (int l = 0; l < d - 1; ++l) M *= n;
    t->M = (int)M;
    t->R_max = R_max;
    t->vt_dev = bf ? (const void *)f.d_Vt16.ptr : (const void *)f.d_Vt32.ptr;
    t->u_dev = bf ? (const void *)f.d_U16.ptr : (const void *)f.d_U32.ptr;
    t->vt_lo_dev = f.d_Vt32lo.ptr;
    t->u_lo_dev = f.d_U32lo.ptr;
    const size_t bytes = (size_t)R_max * M * t->kpad * t->esize;
    // the padding columns are never written: zero them once (the maps read them as K)
    for (DevBuf<uint8_t> *b : {&t->P0, &t->Ta, &t->Tb, &t->P0lo, &t->Talo, &t->Tblo}) {
      if (!t->split && (b == &t->P0lo || b == &t->Talo || b == &t->Tblo)) continue;
      b->alloc(bytes);
      IGA_CUDA_TRY(cudaMemsetAsync(b->ptr, 0, bytes, s));
    }
    t->err.alloc(1);
    IGA_CUDA_TRY(cudaMemsetAsync(t->err.ptr, 0, sizeof(int), s));
    make_map(t->mapP0, t->P0.ptr, bf, n, (long long)R_max * M, t->kpad, kTileM);
    make_map(t->mapTa, t->Ta.ptr, bf, n, (long long)R_max * M, t->kpad, kTileM);
    make_map(t->mapTb, t->Tb.ptr, bf, n, (long long)R_max * M, t->kpad, kTileM);
    if (t->split) {
      make_map(t->mapP0lo, t->P0lo.ptr, 0, n, (long long)R_max * M, t->kpad, kTileM);
      make_map(t->mapTalo, t->Talo.ptr, 0, n, (long long)R_max * M, t->kpad, kTileM);
      make_map(t->mapTblo, t->Tblo.ptr, 0, n, (long long)R_max * M, t->kpad, kTileM);
    }
    t->dinv32 = dinv32;
    // One limit per device, the largest any tile shape needs: the attribute belongs
    // to the kernel, not to this problem, so a smaller per-problem value would
    // invalidate launches already captured by other problems.
    {
      static std::atomic<bool> smem_set[64] = {};
      int dev = 0;
      IGA_CUDA_TRY(cudaGetDevice(&dev));
      const bool done = dev >= 0 && dev < 64 && smem_set[dev].load(std::memory_order_acquire);
      std::unique_lock<DeviceLock> lk(device_mutex(), std::defer_lock);
      if (!done) lk.lock();  // once per device; later setups take no lock here
      if (!done && dev >= 0 && dev < 64 && !smem_set[dev].load(std::memory_order_relaxed)) {
        const int max_smem = 1024 + kStages * (kTileM * 128 + 256 * 128);
        IGA_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<0>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
        IGA_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<1>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
        static_assert(2 * 2 * (kTileM * 128 + 256 * 128) <= kSplitRingBytes,
                      "two split stages of the widest tile fit the ring budget");
        IGA_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<2>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          1024 + kSplitRingBytes));
        {
          const int max_smem_p = (int)(1024 + kTcpRingBytes);
          IGA_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_persistent_kernel<0>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            max_smem_p));
          IGA_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_persistent_kernel<1>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            max_smem_p));
        }
        smem_set[dev].store(true, std::memory_order_release);
      }
    }
    autotune(*t, s);
    IGA_CUDA_TRY(cudaStreamSynchronize(s));
  } catch (...) {
    delete t;
    throw;
  }
  return t;
}

void destroy_tc_fd(TcFd *fd) { delete fd; }

static void gemm(TcFd &t, TcOp Aop, TcOp Bop, const TcEpi &epi, int R, cudaStream_t s) {
  const int M = R * t.M;
  const CUtensorMap &A = *Aop.hi, &B = *Bop.hi;
  if (t.persistent) {
    const long long ntiles = (long long)((M + kTileM - 1) / kTileM) * t.n_ntiles;
    const dim3 pgrid((unsigned)std::min<long long>(ntiles, (long long)num_sms_tc() * t.p_cps));
    if (t.prec == IGA_PREC_BF16)
      launch_pdl(kPdlTensorCore, tc_gemm_persistent_kernel<1>, pgrid, dim3(kTcpThreads),
                 t.p_smem, s, A, B, M, t.n, t.n, t.n_tile, t.tmem_cols, t.idesc, t.p_nstage, epi);
    else
      launch_pdl(kPdlTensorCore, tc_gemm_persistent_kernel<0>, pgrid, dim3(kTcpThreads),
                 t.p_smem, s, A, B, M, t.n, t.n, t.n_tile, t.tmem_cols, t.idesc, t.p_nstage, epi);
    IGA_LAUNCH_CHECK();
    return;
  }
  dim3 grid((M + kTileM - 1) / kTileM, t.n_ntiles);
  if (t.split)
    launch_pdl(kPdlTensorCore, tc_gemm_kernel<2>, grid, dim3(kTcThreads), t.smem, s, A, B,
               *Aop.lo, *Bop.lo, M, t.n, t.n, t.n_tile, t.tmem_cols, t.idesc, epi);
  else if (t.prec == IGA_PREC_BF16)
    launch_pdl(kPdlTensorCore, tc_gemm_kernel<1>, grid, dim3(kTcThreads), t.smem, s, A, B, A, B,
               M, t.n, t.n, t.n_tile, t.tmem_cols, t.idesc, epi);
  else
    launch_pdl(kPdlTensorCore, tc_gemm_kernel<0>, grid, dim3(kTcThreads), t.smem, s, A, B, A, B,
               M, t.n, t.n, t.n_tile, t.tmem_cols, t.idesc, epi);
  IGA_LAUNCH_CHECK();
}

// The chain pack -> d forward products (the d-th fused with the FD diagonal) -> d
// inverse products; the last writes `final` (fp32 or fp64, unpadded, step-indexed).
static void chain(TcFd &t, IdxPtr<const double> in, const TcEpi &final_epi, int R,
                  cudaStream_t s) {
  if (R < 1 || R > t.R_max) throw Error{IGA_ERR_INVALID_ARG, "too many right-hand sides"};
  const bool bf = t.prec == IGA_PREC_BF16;
  const long long N = (long long)R * t.M * t.n;
  if (N > kMaxIndex32) throw Error{IGA_ERR_INVALID_ARG, "more than 2^31 - 1 values per FD apply"};
  const int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 8);
  const FastDiv divn = make_fastdiv((unsigned)t.n);
  if (bf)
    launch_pdl(kPdlTensorCore, pack_kernel<__nv_bfloat16>, dim3(blocks), dim3(256), 0, s, in,
               (__nv_bfloat16 *)t.P0.ptr, (float *)nullptr, (unsigned)N, divn, t.kpad);
  else
    launch_pdl(kPdlTensorCore, pack_kernel<float>, dim3(blocks), dim3(256), 0, s, in,
               (float *)t.P0.ptr, t.split ? (float *)t.P0lo.ptr : (float *)nullptr, (unsigned)N,
               divn, t.kpad);
  IGA_LAUNCH_CHECK();
  TcEpi mid{};
  mid.kind = bf ? kOutBF16 : kOutF32;
  mid.tf32_round = bf ? 0 : 1;
  mid.n = t.n;
  mid.ld_out = t.kpad;
  mid.nmid = t.M / t.n;
  mid.err = t.err.ptr;
  auto to = [&](int which) {
    TcEpi e = mid;
    e.out = which ? t.Tb.ptr : t.Ta.ptr;
    if (t.split) e.out_lo = (float *)(which ? t.Tblo.ptr : t.Talo.ptr);
    return e;
  };
  TcOp cur{&t.mapP0, &t.mapP0lo};
  const TcOp maps[2] = {{&t.mapTa, &t.mapTalo}, {&t.mapTb, &t.mapTblo}};
  int which = 0;
  const int total = 2 * t.d;
  for (int g = 0; g < total; ++g) {
    const bool fwd = g < t.d;
    const TcOp B = fwd ? TcOp{&t.mapVt, &t.mapVtlo} : TcOp{&t.mapU, &t.mapUlo};
    TcEpi e;
    if (g == total - 1) {
      e = final_epi;
    } else {
      e = to(which);
    }
    if (g == t.d - 1) {
      e.dinv = t.dinv32;
    }
    gemm(t, cur, B, e, R, s);
    if (g != total - 1) {
      cur = maps[which];
      which ^= 1;
    }
  }
}

void tc_fd_apply(TcFd &t, IdxPtr<const double> in, IdxPtr<float> out, int R, cudaStream_t s) {
  TcEpi e{};
  e.out = out.base;
  e.oidx = out.idx;
  e.ostride = out.stride;
  if (out.idx) e.ostride = out.stride;
  e.kind = kOutF32;
  e.tf32_round = 0;
  e.n = t.n;
  e.ld_out = t.n;
  e.nmid = t.M / t.n;
  e.err = t.err.ptr;
  if (out.idx && out.off) throw Error{IGA_ERR_INVALID_ARG, "unsupported output offset"};
  chain(t, in, e, R, s);
}

void tc_fd_apply_f64out(TcFd &t, IdxPtr<const double> in, double *out, int R, cudaStream_t s) {
  TcEpi e{};
  e.out = out;
  e.kind = kOutF64;
  e.n = t.n;
  e.ld_out = t.n;
  e.nmid = t.M / t.n;
  e.err = t.err.ptr;
  chain(t, in, e, R, s);
}

int *tc_fd_error_word(TcFd &t) { return t.err.ptr; }

void preload_kernels_fd_tc() {
  cudaFuncAttributes a;
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, tc_gemm_kernel<0>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, tc_gemm_kernel<1>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, tc_gemm_kernel<2>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, tc_gemm_persistent_kernel<0>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, tc_gemm_persistent_kernel<1>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, pack_kernel<float>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, pack_kernel<__nv_bfloat16>));
}

}  // namespace iga
