// GMRES kernels for R right-hand sides in lockstep: deterministic reductions,
// classical Gram-Schmidt with one re-orthogonalization (CGS2) as batched GEMV passes
// with fused norms, Givens rotations of the Hessenberg column, back substitution and
// the solution update.
//
// The Krylov method is GMRES (Saad & Schultz, named in Sec. 3 of the paper).  Each
// right-hand side r has its own Krylov basis V_r, Hessenberg matrix, rotations and
// convergence flag; all share the step number k in device memory (SolveState::k) so
// that one CUDA graph replays every iteration.  A right-hand side that has converged
// is frozen: the reduction kernels skip it and its step count stays put.
// Reductions over blocks are done by the last block to finish (atomic ticket, no
// spinning), always in block order, so results are bitwise reproducible, and the
// same for a right-hand side alone or among others.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "contract_point.cuh"
#include "fp_widen.h"
#include "iga_internal.h"

namespace iga {

constexpr int kRT = 256;  // threads per reduction block
constexpr int kWarps = kRT / 32;
constexpr int kJC = 8;    // vectors per register chunk

// Grid of the reduction passes.  It depends on N and the handle's grid mode only, so
// that the row partition -- and with it the order of every reduction -- is the same for
// a right-hand side alone or among others; each block loops over the right-hand sides.
// Measured on GB300: for one solve at a time two blocks per SM (eight warps each) work
// best, more blocks make the last-block reduction over their partials slower than they
// gain (latency mode, >= 512 rows a block); with many solves running at once (batched
// form, 256 problems x 8 right-hand sides) a block per 4096 rows, at most one per SM,
// gives 27 % more throughput (throughput mode).
int reduce_blocks(long long N, int mode) {
  static int sms = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 152;
    return n;
  }();
  const long long rows = mode == IGA_GRID_THROUGHPUT ? 4096 : 512;
  const long long cap = mode == IGA_GRID_THROUGHPUT ? sms : 2LL * sms;
  long long b = (N + rows - 1) / rows;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

__device__ __forceinline__ void row_range(long long N, long long &lo, long long &hi) {
  const long long chunk = (N + gridDim.x - 1) / gridDim.x;
  lo = (long long)blockIdx.x * chunk;
  hi = min(N, lo + chunk);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp reduction of 8 accumulators at once by halving exchange: at offsets 16, 8, 4
// each lane keeps half of its remaining values and adds the partner's matching half,
// then offsets 2 and 1 finish the sum.  9 FP64 adds per lane instead of 8 x 5.  On
// return lane l holds the warp total of accumulator ((l>>4)&1)*4 + ((l>>3)&1)*2 +
// ((l>>2)&1).
__device__ __forceinline__ double warp_reduce8(const double (&a)[kJC]) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  double b4[4], b2[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double keep = h16 ? a[q + 4] : a[q];
    const double send = h16 ? a[q] : a[q + 4];
    b4[q] = keep + __shfl_xor_sync(full, send, 16);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double keep = h8 ? b4[q + 2] : b4[q];
    const double send = h8 ? b4[q] : b4[q + 2];
    b2[q] = keep + __shfl_xor_sync(full, send, 8);
  }
  double v = (h4 ? b2[1] : b2[0]) + __shfl_xor_sync(full, h4 ? b2[0] : b2[1], 4);
  v += __shfl_xor_sync(full, v, 2);
  v += __shfl_xor_sync(full, v, 1);
  return v;
}

// Block-reduce acc[0..cnt) and store partial[(j0+q)*nblk + blockIdx.x].
__device__ __forceinline__ void block_store_partials(double (&acc)[kJC], int cnt, int j0,
                                                     double *partial, int nblk,
                                                     double (*red)[kJC]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double v = warp_reduce8(acc);
  if ((lane & 3) == 0) red[warp][((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)] = v;
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
    partial[(long long)(j0 + threadIdx.x) * nblk + blockIdx.x] = s;
  }
  __syncthreads();
}

// True in exactly one block of the row (the last to arrive); that block then sees
// every other block's partials.
__device__ __forceinline__ bool arrive_last(unsigned int *counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Sum partial[j*nblk + b] over b (fixed order) for j < cnt into out[j] (op 0: store,
// 1: add); optionally also store the sums in out2[j].  tail (optional): the last row,
// j = cnt - 1, is stored there instead (op and out2 do not apply to it), so that one call
// reduces a pass's coefficients and its norm together.
// A lane loads all of its partials of a row (up to kLdPer per round) before it adds them,
// in the same order as one add per load: a row costs one L2 round trip per 32 kLdPer
// partials.  Loaded and added one at a time they cost one round trip per 32, which made
// the single last block's reduction the largest fixed cost of a pass (~20 us per CGS2
// pass 2 at 2.2e6 rows with 304 blocks, two reductions in series).
constexpr int kLdPer = 10;
__device__ void last_block_reduce(const double *partial, int nblk, int cnt, double *out, int op,
                                  double *out2, double *tail = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < cnt; j += kWarps) {
    const double *pj = partial + (long long)j * nblk;
    double s = 0.0;
    for (int b0 = 0; b0 < nblk; b0 += 32 * kLdPer) {
      double t[kLdPer];
#pragma unroll
      for (int q = 0; q < kLdPer; ++q) {
        const int b = b0 + lane + 32 * q;
        t[q] = b < nblk ? __ldcg(pj + b) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < kLdPer; ++q) s += t[q];
    }
    s = warp_sum(s);
    if (lane == 0) {
      if (tail && j == cnt - 1) {
        *tail = s;
      } else {
        if (op == 0) out[j] = s; else out[j] += s;
        if (out2) out2[j] = s;
      }
    }
  }
}

__device__ __forceinline__ long long ldh(const KrylovWs &ws) { return ws.max_iter + 1; }
__device__ __forceinline__ double *Hcol(const KrylovWs &ws, int r, int k) {
  return ws.H + r * ws.hstride + ldh(ws) * k;
}
__device__ __forceinline__ const double *Vvec(const KrylovWs &ws, int j, int r) {
  return ws.V + ((long long)j * ws.R + r) * ws.N;
}

// ------------------------------------------------------------------ init
// ||b_r||^2 -> scal[8r], ||r0_r||^2 -> scal[8r+1]
__global__ void __launch_bounds__(kRT) init_norms_kernel(KrylovWs ws, const double *__restrict__ b,
                                                         const double *__restrict__ r0) {
  __shared__ double red[kWarps][kJC];
  const int r = blockIdx.y;
  const double *br = b + (long long)r * ws.N, *rr = r0 + (long long)r * ws.N;
  long long lo, hi;
  row_range(ws.N, lo, hi);
  double acc[kJC] = {};
  for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
    acc[0] = fma(br[i], br[i], acc[0]);
    acc[1] = fma(rr[i], rr[i], acc[1]);
  }
  double *part = ws.partials + r * ws.pstride;
  block_store_partials(acc, 2, 0, part, gridDim.x, red);
  if (!arrive_last(ws.counter + r)) return;
  last_block_reduce(part, gridDim.x, 2, ws.scal + 8 * r, 0, nullptr);
  __syncthreads();
  if (threadIdx.x == 0) ws.counter[r] = 0;
}

__global__ void init_finalize_kernel(KrylovWs ws, cudaGraphConditionalHandle cond, int has_cond) {
  __shared__ int active;
  if (threadIdx.x == 0) active = 0;
  __syncthreads();
  SolveState *st = ws.st;
  for (int r = threadIdx.x; r < ws.R; r += blockDim.x) {
    RhsState &q = ws.rs[r];
    const double bn = sqrt(ws.scal[8 * r]);
    const double beta = sqrt(ws.scal[8 * r + 1]);
    q.bnorm = bn;
    q.beta = beta;
    q.kconv = 0;
    q.relres_true = 0.0;
    ws.g[r * (ws.max_iter + 2)] = beta;
    ws.hist[r * (ws.max_iter + 2)] = bn > 0.0 ? beta / bn : 0.0;
    int done = 0, flag = 0;
    if (!isfinite(bn) || !isfinite(beta)) {
      done = 1;
      flag = 4;
    } else if (beta == 0.0 || beta <= st->tol * bn) {
      done = 1;
      flag = 1;
    } else if (st->max_iter <= 0) {
      done = 1;
      flag = 2;
    }
    q.done = done;
    q.flag = flag;
    if (!done) atomicAdd(&active, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->k = 0;
    st->active = active;
    if (has_cond) cudaGraphSetConditional(cond, active > 0 ? 1u : 0u);
  }
}

__global__ void scale_v0_kernel(KrylovWs ws, const double *__restrict__ r0) {
  const int r = blockIdx.y;
  const RhsState &q = ws.rs[r];
  const double inv = q.done ? 0.0 : 1.0 / q.beta;
  double *v = ws.V + (long long)r * ws.N;
  const double *src = r0 + (long long)r * ws.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ws.N;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = src[i] * inv;
}

void launch_init_solve(const KrylovWs &ws, const double *b, const double *r0,
                       cudaGraphConditionalHandle cond, int has_cond, cudaStream_t s) {
  init_norms_kernel<<<dim3(ws.nblk, ws.R), kRT, 0, s>>>(ws, b, r0);
  IGA_LAUNCH_CHECK();
  init_finalize_kernel<<<1, 256, 0, s>>>(ws, cond, has_cond);
  IGA_LAUNCH_CHECK();
  scale_v0_kernel<<<dim3(ws.nblk, ws.R), kRT, 0, s>>>(ws, r0);
  IGA_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ CGS2
// The passes are bound by the FP64 unit (one FMA per vector entry read, against an FP64
// rate of about 0.5 FMA per clock per SM sub-partition), with the memory traffic close
// behind: every warp must keep loads in flight while its FMAs issue.  The loops below
// therefore load the next step's operands before they issue the current step's FMAs.

// Exact counts.  A predicated-off FP64 instruction still takes its issue slot on GB300's
// narrow FP64 unit (ncu: the passes ran the unit 85-88 % busy while doing 72-78 % useful
// FMAs), so every loop over a runtime count of vectors or outputs is compiled for its exact
// count (a template argument, chosen by a warp-uniform switch) instead of a fixed maximum
// with a predicate.

// Dots of vectors V_r[j0 .. j0+CNT) with u over this block's rows, one row per thread and
// step, the next step's entries loaded before this step's FMAs (rows past the block's end
// read as zero, which adds exact zeros); block-reduced into partials.  Index jself (if in
// range) stands for u itself: its dot is ||u||^2 over the rows.
template <int CNT>
__device__ __forceinline__ void chunk_dots_n(const KrylovWs &ws, int r, int j0,
                                             const double *__restrict__ u, long long lo,
                                             long long hi, double *part, double (*red)[kJC],
                                             int jself) {
  const double *vb[CNT];
#pragma unroll
  for (int q = 0; q < CNT; ++q) {
    const int j = j0 + q;
    vb[q] = j == jself ? u : Vvec(ws, j, r);
  }
  double acc[kJC] = {};
  double u0, a0[CNT];
  auto load = [&](long long i, double &x, double (&b)[CNT]) {
    const bool ok = i < hi;
    x = ok ? u[i] : 0.0;
#pragma unroll
    for (int q = 0; q < CNT; ++q) b[q] = ok ? vb[q][i] : 0.0;
  };
  long long i = lo + threadIdx.x;
  load(i, u0, a0);
  for (; i < hi; i += kRT) {
    double nu, n0[CNT];
    load(i + kRT, nu, n0);
#pragma unroll
    for (int q = 0; q < CNT; ++q) acc[q] = fma(a0[q], u0, acc[q]);
    u0 = nu;
#pragma unroll
    for (int q = 0; q < CNT; ++q) a0[q] = n0[q];
  }
  block_store_partials(acc, CNT, j0, part, gridDim.x, red);
}

__device__ __forceinline__ void chunk_dots(const KrylovWs &ws, int r, int j0, int cnt,
                                           const double *__restrict__ u, long long lo,
                                           long long hi, double *part, double (*red)[kJC],
                                           int jself = -1) {
  switch (cnt) {
    case 1: chunk_dots_n<1>(ws, r, j0, u, lo, hi, part, red, jself); break;
    case 2: chunk_dots_n<2>(ws, r, j0, u, lo, hi, part, red, jself); break;
    case 3: chunk_dots_n<3>(ws, r, j0, u, lo, hi, part, red, jself); break;
    case 4: chunk_dots_n<4>(ws, r, j0, u, lo, hi, part, red, jself); break;
    case 5: chunk_dots_n<5>(ws, r, j0, u, lo, hi, part, red, jself); break;
    case 6: chunk_dots_n<6>(ws, r, j0, u, lo, hi, part, red, jself); break;
    case 7: chunk_dots_n<7>(ws, r, j0, u, lo, hi, part, red, jself); break;
    default: chunk_dots_n<8>(ws, r, j0, u, lo, hi, part, red, jself); break;
  }
}

// u[i] - (V_r h)[i] and the same for row i + kRT, as one FMA chain per row that starts at u
// (rows past hi read as zero): on GB300 a warp-wide FP64 FMA holds a sub-partition's FP64
// unit for ~64 cycles, so one chain per row with four warps per sub-partition keeps the
// unit busy, and the chain needs no adds to combine partial sums (split accumulators
// cost 2 FP64 adds per row).  kPG vectors' entries are loaded ahead of their FMAs.
constexpr int kPG = 3;
__device__ __forceinline__ void sub_proj_rows(const KrylovWs &ws, int r, int nv,
                                              const double *__restrict__ hs, long long i,
                                              long long hi, double &x0, double &x1) {
  const bool v0 = i < hi, v1 = i + kRT < hi;
  double c0[kPG], c1[kPG];
  const int full = nv - nv % kPG;
  auto load = [&](int j, double (&b0)[kPG], double (&b1)[kPG]) {
#pragma unroll
    for (int q = 0; q < kPG; ++q) {
      const double *v = Vvec(ws, j + q, r);
      b0[q] = v0 ? v[i] : 0.0;
      b1[q] = v1 ? v[i + kRT] : 0.0;
    }
  };
  if (full > 0) load(0, c0, c1);
  for (int j = 0; j < full; j += kPG) {
    double n0[kPG], n1[kPG];
    if (j + kPG < full) load(j + kPG, n0, n1);
#pragma unroll
    for (int q = 0; q < kPG; ++q) {
      x0 = fma(-c0[q], hs[j + q], x0);
      x1 = fma(-c1[q], hs[j + q], x1);
    }
#pragma unroll
    for (int q = 0; q < kPG; ++q) {
      c0[q] = n0[q];
      c1[q] = n1[q];
    }
  }
  for (int j = full; j < nv; ++j) {  // nv mod kPG <= 2 vectors
    const double *v = Vvec(ws, j, r);
    x0 = fma(-(v0 ? v[i] : 0.0), hs[j], x0);
    x1 = fma(-(v1 ? v[i + kRT] : 0.0), hs[j], x1);
  }
}

// dst[i] = (u_r[i] - sum_j V_r[j][i] h[j]) (* scale with kScale) for this block's rows.
// dst may be u.  hs: the nv coefficients in shared memory.
template <bool kScale = false>
__device__ __forceinline__ void subtract_proj(const KrylovWs &ws, int r, int nv,
                                              const double *__restrict__ hs, const double *u,
                                              long long lo, long long hi, double *dst,
                                              double scale = 1.0) {
  for (long long i = lo + threadIdx.x; i < hi; i += 2 * kRT) {
    double x0 = u[i], x1 = i + kRT < hi ? u[i + kRT] : 0.0;
    sub_proj_rows(ws, r, nv, hs, i, hi, x0, x1);
    if (kScale) x0 *= scale;
    dst[i] = x0;
    if (i + kRT < hi) {
      if (kScale) x1 *= scale;
      dst[i + kRT] = x1;
    }
  }
}

// Pass 2 for NV = nv <= 15 vectors, reading V_r from memory once: per row, the NV entries
// of V_r are loaded, w' = w - V_r h1 as one FMA chain, then the dots of V_r and w' with w'
// from the same registers, NV + 1 accumulators over the block's rows.  The other warps of
// the sub-partition cover the loads' latency (each row is 2 NV + 1 warp FMAs, ~64 cycles
// of the FP64 unit apiece).
template <int NV>
__device__ __forceinline__ void pass2_fused(const KrylovWs &ws, int r,
                                            const double *__restrict__ hs, double *w,
                                            long long lo, long long hi, double *part,
                                            double (*red)[kJC]) {
  constexpr int NA = (NV + 1 + kJC - 1) / kJC * kJC;
  double acc[NA] = {};
  const long long vs = (long long)ws.R * ws.N;  // stride between V_r[j] and V_r[j + 1]
  const double *__restrict__ v0 = Vvec(ws, 0, r);
  for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
    double b[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) b[j] = v0[i + j * vs];
    double x = w[i];
#pragma unroll
    for (int j = 0; j < NV; ++j) x = fma(-b[j], hs[j], x);
    w[i] = x;
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = fma(b[j], x, acc[j]);
    acc[NV] = fma(x, x, acc[NV]);
  }
#pragma unroll
  for (int c = 0; c < NA / kJC; ++c) {
    double a[kJC];
#pragma unroll
    for (int q = 0; q < kJC; ++q) a[q] = acc[c * kJC + q];
    block_store_partials(a, min(kJC, NV + 1 - c * kJC), c * kJC, part, gridDim.x, red);
  }
}

// Pass 2 for 15 < NV = nv <= kStashMax vectors, still reading V_r once: the row's NV
// entries are too many to keep in registers beside the NV + 1 accumulators, so the chain
// w' = w - V_r h1 stores each entry it loads into this thread's column of shared memory
// (stash[j * kRT + thread]) and the dots read them back from there.  The same FMAs in the
// same order as subtract_proj followed by chunk_dots (the path for more vectors), and the
// same partials, so both give bitwise the same w', h2 and norm.  Measured at 2.2e6 rows
// (the 3D 128-element annulus), 16 vectors: the two-sweep path took 38 us more than 15
// vectors in one sweep, this one 12 us more (16..21 vectors: 26-32 us less than the
// two-sweep path).
// 24 and more spill registers (NA = 32 accumulators); 22 and 23 measured slower than 16..21
// (the 3D 128-element annulus: 23 vectors took 306 us against 226 us on the two-sweep path)
constexpr int kStashMax = 21;
template <int NV>
__device__ __forceinline__ void pass2_stash(const KrylovWs &ws, int r,
                                            const double *__restrict__ hs, double *w,
                                            long long lo, long long hi, double *part,
                                            double (*red)[kJC], double *stash) {
  constexpr int NA = (NV + 1 + kJC - 1) / kJC * kJC;
  double acc[NA] = {};
  const long long vs = (long long)ws.R * ws.N;
  const double *__restrict__ v0 = Vvec(ws, 0, r);
  double *st = stash + threadIdx.x;
  for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
    double x = w[i];
    // loads in groups of kJC: the compiler barrier after each group's stash stores keeps
    // it from hoisting all NV loads above the chain (NV + NA live doubles spilled)
#pragma unroll
    for (int j0 = 0; j0 < NV; j0 += kJC) {
#pragma unroll
      for (int j = j0; j < j0 + kJC && j < NV; ++j) {
        const double b = v0[i + j * vs];
        x = fma(-b, hs[j], x);
        st[j * kRT] = b;
      }
      asm volatile("" ::: "memory");
    }
    w[i] = x;
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = fma(st[j * kRT], x, acc[j]);
    acc[NV] = fma(x, x, acc[NV]);
  }
#pragma unroll
  for (int c = 0; c < NA / kJC; ++c) {
    double a[kJC];
#pragma unroll
    for (int q = 0; q < kJC; ++q) a[q] = acc[c * kJC + q];
    block_store_partials(a, min(kJC, NV + 1 - c * kJC), c * kJC, part, gridDim.x, red);
  }
}

// Whether pass 2 takes pass2_stash for 15 < nv <= kStashMax (IGA_P2_STASH=0: the
// two-sweep path, to check that both give the same bits).
static bool p2_stash() {
  static const bool on = [] {
    const char *e = std::getenv("IGA_P2_STASH");
    return !(e && e[0] == '0');
  }();
  return on;
}

// Dynamic shared memory of pass 2: the max_iter + 1 coefficients and, when a step can
// have more than 15 basis vectors, the stash of pass2_stash.
static bool pass2_has_stash(int max_iter) { return p2_stash() && max_iter + 1 > 15; }
static size_t pass2_smem(int max_iter, bool stash) {
  return (size_t)(max_iter + 1) * sizeof(double) +
         (stash ? (size_t)kStashMax * kRT * sizeof(double) : 0);
}

// Pass 1 for NV = nv <= 15 vectors: the dots of V_r with w over the block's rows in one
// sweep (w read once), NV accumulators in registers.
template <int NV>
__device__ __forceinline__ void pass1_fused(const KrylovWs &ws, int r,
                                            const double *__restrict__ w, long long lo,
                                            long long hi, double *part, double (*red)[kJC]) {
  constexpr int NA = (NV + kJC - 1) / kJC * kJC;
  double acc[NA] = {};
  const long long vs = (long long)ws.R * ws.N;
  const double *__restrict__ v0 = Vvec(ws, 0, r);
  for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
    double b[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) b[j] = v0[i + j * vs];
    const double u = w[i];
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = fma(b[j], u, acc[j]);
  }
#pragma unroll
  for (int c = 0; c < NA / kJC; ++c) {
    double a[kJC];
#pragma unroll
    for (int q = 0; q < kJC; ++q) a[q] = acc[c * kJC + q];
    block_store_partials(a, min(kJC, NV - c * kJC), c * kJC, part, gridDim.x, red);
  }
}

// pass 1: h1 = V_r^T w_r -> H_r[0..k, k]
__global__ void __launch_bounds__(kRT, 2) cgs_pass1_kernel(KrylovWs ws, const double *__restrict__ w) {
  pdl_entry();
  __shared__ double red[kWarps][kJC];
  const int k = ws.st->k, nv = k + 1;
  long long lo, hi;
  row_range(ws.N, lo, hi);
  for (int r = 0; r < ws.R; ++r) {
    if (ws.rs[r].done) continue;
    const double *wr = w + (long long)r * ws.N;
    double *part = ws.partials + r * ws.pstride;
#define IGA_P1(NVV) \
  case NVV: pass1_fused<NVV>(ws, r, wr, lo, hi, part, red); break;
    switch (nv) {
      IGA_P1(1) IGA_P1(2) IGA_P1(3) IGA_P1(4) IGA_P1(5) IGA_P1(6) IGA_P1(7) IGA_P1(8) IGA_P1(9) IGA_P1(10) IGA_P1(11) IGA_P1(12) IGA_P1(13) IGA_P1(14) IGA_P1(15)
      default:
        for (int j0 = 0; j0 < nv; j0 += kJC)
          chunk_dots(ws, r, j0, min(kJC, nv - j0), wr, lo, hi, part, red);
    }
#undef IGA_P1
    if (!arrive_last(ws.counter + r)) continue;
    last_block_reduce(part, gridDim.x, nv, Hcol(ws, r, k), 0, nullptr);
    __syncthreads();
    if (threadIdx.x == 0) ws.counter[r] = 0;
  }
}

// Pass 1 fused with the operator's last pass, for NV = nv <= 15 vectors: per row, w is
// contracted (contract_point), stored, and dotted with the row's NV entries of V_r; the
// same FMAs in the same order as contract_pass_kernel followed by pass1_fused.
template <int W, int NV>
__device__ __forceinline__ void pass1_op_fused(const KrylovWs &ws, int r,
                                               const ContractArgsT<double> &a, const BandDev &b,
                                               const FastDiv &divn, double *wr, long long lo,
                                               long long hi, double *part, double (*red)[kJC]) {
  constexpr int NA = (NV + kJC - 1) / kJC * kJC;
  double acc[NA] = {};
  const long long vs = (long long)ws.R * ws.N;
  const double *__restrict__ v0 = Vvec(ws, 0, r);
  const long long roff = (long long)r * ws.N;
  for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
    const int c = (int)((unsigned)i - fdiv((unsigned)i, divn) * divn.d);
    const double u = contract_point<double, W>(a, roff + i, (unsigned)i, c, b);
    wr[i] = u;
    double bb[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) bb[j] = v0[i + j * vs];
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = fma(bb[j], u, acc[j]);
  }
#pragma unroll
  for (int c = 0; c < NA / kJC; ++c) {
    double t[kJC];
#pragma unroll
    for (int q = 0; q < kJC; ++q) t[q] = acc[c * kJC + q];
    block_store_partials(t, min(kJC, NV - c * kJC), c * kJC, part, gridDim.x, red);
  }
}

// the operator's last pass (w for this block's rows of right-hand side r) fused with pass 1
template <int W>
__global__ void __launch_bounds__(kRT, 2)
    cgs_pass1_op_kernel(KrylovWs ws, ContractArgsT<double> a, BandDev b, FastDiv divn,
                        double *w) {
  pdl_entry();
  __shared__ double red[kWarps][kJC];
  const int k = ws.st->k, nv = k + 1;
  long long lo, hi;
  row_range(ws.N, lo, hi);
  for (int r = 0; r < ws.R; ++r) {
    if (ws.rs[r].done) continue;
    double *wr = w + (long long)r * ws.N;
    double *part = ws.partials + r * ws.pstride;
#define IGA_P1OP(NVV) \
  case NVV: pass1_op_fused<W, NVV>(ws, r, a, b, divn, wr, lo, hi, part, red); break;
    switch (nv) {
      IGA_P1OP(1) IGA_P1OP(2) IGA_P1OP(3) IGA_P1OP(4) IGA_P1OP(5) IGA_P1OP(6) IGA_P1OP(7) IGA_P1OP(8) IGA_P1OP(9) IGA_P1OP(10) IGA_P1OP(11) IGA_P1OP(12) IGA_P1OP(13) IGA_P1OP(14) IGA_P1OP(15)
      default: {
        const long long roff = (long long)r * ws.N;
        for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
          const int c = (int)((unsigned)i - fdiv((unsigned)i, divn) * divn.d);
          wr[i] = contract_point<double, W>(a, roff + i, (unsigned)i, c, b);
        }
        __syncthreads();  // the block's rows of w are complete (and visible) for the dots
        for (int j0 = 0; j0 < nv; j0 += kJC)
          chunk_dots(ws, r, j0, min(kJC, nv - j0), wr, lo, hi, part, red);
      }
    }
#undef IGA_P1OP
    if (!arrive_last(ws.counter + r)) continue;
    last_block_reduce(part, gridDim.x, nv, Hcol(ws, r, k), 0, nullptr);
    __syncthreads();
    if (threadIdx.x == 0) ws.counter[r] = 0;
  }
}

// pass 2: w_r -= V_r h1; h2 = V_r^T w_r -> H_r[0..k,k] += h2, y_r = h2; nu = ||w_r||^2;
// H_r[k+1,k] = sqrt(nu - ||h2||^2), the norm of w_r - V_r h2 (V_r orthonormal), so
// that pass 3 needs no reduction of its own.  After the first projection w_r is
// orthogonal to V_r to working accuracy, ||h2|| <= ||w_r|| times a small multiple of the
// unit roundoff, and the difference loses no significant digits.
// stash: the dynamic shared memory holds pass2_stash's buffer (15 < nv <= kStashMax runs
// pass2_stash; otherwise more than 15 vectors take the two-sweep path).
__global__ void __launch_bounds__(kRT, 2) cgs_pass2_kernel(KrylovWs ws, double *__restrict__ w,
                                                           int stash_on) {
  pdl_entry();
  __shared__ double red[kWarps][kJC];
  extern __shared__ double hs[];  // max_iter + 1 coefficients, then the stash (pass2_smem)
  double *stash = hs + (ws.max_iter + 1);
  const int k = ws.st->k, nv = k + 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) ws.st->kv = k;
  long long lo, hi;
  row_range(ws.N, lo, hi);
  for (int r = 0; r < ws.R; ++r) {
    if (ws.rs[r].done) continue;
    double *wr = w + (long long)r * ws.N;
    const double *h1 = Hcol(ws, r, k);
    double *part = ws.partials + r * ws.pstride;
    __syncthreads();  // hs of the previous right-hand side is no longer read
    for (int j = threadIdx.x; j < nv; j += kRT) hs[j] = h1[j];
    __syncthreads();
#define IGA_P2(NVV) \
  case NVV: pass2_fused<NVV>(ws, r, hs, wr, lo, hi, part, red); break;
#define IGA_P2S(NVV) \
  case NVV: pass2_stash<NVV>(ws, r, hs, wr, lo, hi, part, red, stash); break;
    switch (nv > 15 && !stash_on ? 0 : nv) {
      IGA_P2(1) IGA_P2(2) IGA_P2(3) IGA_P2(4) IGA_P2(5) IGA_P2(6) IGA_P2(7) IGA_P2(8) IGA_P2(9) IGA_P2(10) IGA_P2(11) IGA_P2(12) IGA_P2(13) IGA_P2(14) IGA_P2(15)
      IGA_P2S(16) IGA_P2S(17) IGA_P2S(18) IGA_P2S(19) IGA_P2S(20) IGA_P2S(21)
      default:
        subtract_proj(ws, r, nv, hs, wr, lo, hi, wr);
        for (int j0 = 0; j0 <= nv; j0 += kJC)
          chunk_dots(ws, r, j0, min(kJC, nv + 1 - j0), wr, lo, hi, part, red, nv);
    }
#undef IGA_P2
#undef IGA_P2S
    if (!arrive_last(ws.counter + r)) continue;
    double *y = ws.y + r * (ws.max_iter + 2);
    // the nv coefficients h2 and, as row nv, ||w_r||^2
    last_block_reduce(part, gridDim.x, nv + 1, Hcol(ws, r, k), 1, y, ws.scal + 8 * r + 2);
    __syncthreads();
    if (threadIdx.x < 32) {
      double q = 0.0;
      for (int j = threadIdx.x; j < nv; j += 32) q = fma(y[j], y[j], q);
      q = warp_sum(q);
      if (threadIdx.x == 0) {
        const double b2 = ws.scal[8 * r + 2] - q;
        const double beta = b2 > 0.0 ? sqrt(b2) : 0.0;
        Hcol(ws, r, k)[k + 1] = beta;  // the Givens kernel rotates this entry away
        ws.scal[8 * r + 4] = beta;     // pass 3 reads this copy
        ws.counter[r] = 0;
      }
    }
  }
}

// pass 3: v_{k+1} = (w_r - V_r h2) / H_r[k+1,k] (zero on breakdown).  It runs beside the
// Givens kernel of the same step, which advances k, sets the done flags and rotates H:
// the step comes from kv and the norm from its copy in scal.  A right-hand side that the
// Givens kernel has just retired may or may not get its v_{k+1}; it is never read.
__global__ void __launch_bounds__(kRT, 2) cgs_pass3_kernel(KrylovWs ws, const double *__restrict__ w) {
  pdl_entry();
  extern __shared__ double hs[];  // max_iter + 1 coefficients
  const int k = ws.st->kv, nv = k + 1;
  long long lo, hi;
  row_range(ws.N, lo, hi);
  for (int r = 0; r < ws.R; ++r) {
    if (ws.rs[r].done) continue;
    const double *wr = w + (long long)r * ws.N;
    const double *h2 = ws.y + r * (ws.max_iter + 2);
    __syncthreads();
    for (int j = threadIdx.x; j < nv; j += kRT) hs[j] = h2[j];
    __syncthreads();
    const double hn = ws.scal[8 * r + 4];
    const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
    double *v = ws.V + ((long long)(k + 1) * ws.R + r) * ws.N;
    subtract_proj<true>(ws, r, nv, hs, wr, lo, hi, v, inv);
  }
}

void launch_cgs2_coeffs(const KrylovWs &ws, double *w, cudaStream_t s) {
  const dim3 grid(ws.nblk);
  launch_pdl(kPdlKrylov, cgs_pass1_kernel, grid, dim3(kRT), 0, s, ws, (const double *)w);
  IGA_LAUNCH_CHECK();
  const bool st = pass2_has_stash(ws.max_iter);
  launch_pdl(kPdlKrylov, cgs_pass2_kernel, grid, dim3(kRT), pass2_smem(ws.max_iter, st), s, ws, w,
             st ? 1 : 0);
  IGA_LAUNCH_CHECK();
}

void launch_cgs2_pass2(const KrylovWs &ws, double *w, cudaStream_t s) {
  const bool st = pass2_has_stash(ws.max_iter);
  launch_pdl(kPdlKrylov, cgs_pass2_kernel, dim3(ws.nblk), dim3(kRT), pass2_smem(ws.max_iter, st),
             s, ws, w, st ? 1 : 0);
  IGA_LAUNCH_CHECK();
}

void launch_cgs_pass1_op(const KrylovWs &ws, const ContractArgsT<double> &a, const BandDev &b,
                         int n, double *w, cudaStream_t s) {
  const FastDiv divn = make_fastdiv((unsigned)n);
  const dim3 grid(ws.nblk);
  switch (b.W) {
#define IGA_P1OP_W(WW)                                                                      \
  case WW:                                                                                   \
    launch_pdl(kPdlKrylov, cgs_pass1_op_kernel<WW>, grid, dim3(kRT), 0, s, ws, a, b, divn, w); \
    break;
    IGA_P1OP_W(3) IGA_P1OP_W(4) IGA_P1OP_W(5) IGA_P1OP_W(6) IGA_P1OP_W(7)
#undef IGA_P1OP_W
    default:
      throw Error{IGA_ERR_INVALID_ARG, "band width out of range"};
  }
  IGA_LAUNCH_CHECK();
}

bool fuse_pass1() {
  static const bool on = [] {
    const char *e = std::getenv("IGA_FUSE_P1");
    return !(e && e[0] == '0');
  }();
  return on;
}

void launch_cgs2_vector(const KrylovWs &ws, const double *w, cudaStream_t s) {
  launch_pdl(kPdlKrylov, cgs_pass3_kernel, dim3(ws.nblk), dim3(kRT),
             (ws.max_iter + 1) * sizeof(double), s, ws, w);
  IGA_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ Givens
__device__ void givens_cs(double a, double b, double &c, double &s) {
  if (b == 0.0) {
    c = 1.0;
    s = 0.0;
  } else if (fabs(b) > fabs(a)) {
    const double t = a / b;
    s = 1.0 / sqrt(1.0 + t * t);
    c = s * t;
  } else {
    const double t = b / a;
    c = 1.0 / sqrt(1.0 + t * t);
    s = c * t;
  }
}

constexpr int kGC = 128;  // rotations staged in shared memory per pass

// For every live right-hand side (one warp each): rotate column k of H by the previous
// rotations, build rotation k, update g and the residual estimate, decide convergence.
// Then advance k and continue the loop while any right-hand side is live.  The
// rotations and the column are staged in shared memory by the whole warp first, so
// the sequential recurrence (carried in a register) waits on no global loads.
__global__ void givens_kernel(KrylovWs ws, cudaGraphConditionalHandle cond, int has_cond) {
  __shared__ int active;
  __shared__ double sh_cs[4][kGC], sh_sn[4][kGC], sh_b[4][kGC];
  pdl_entry();
  SolveState *st = ws.st;
  const int k = st->k;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) active = 0;
  __syncthreads();
  for (int r = warp; r < ws.R; r += nwarps) {
    RhsState &q = ws.rs[r];
    if (q.done) continue;
    double *col = Hcol(ws, r, k);
    double *cs = ws.cs + r * (ws.max_iter + 1), *sn = ws.sn + r * (ws.max_iter + 1);
    double *g = ws.g + r * (ws.max_iter + 2);
    const double hk1 = col[k + 1];
    // t carries the rotated entry i (the "a" of rotation i); b = original entry i+1
    double t = col[0];
    for (int base = 0; base < k; base += kGC) {
      const int m = min(kGC, k - base);
      for (int e = lane; e < m; e += 32) {
        sh_cs[warp][e] = cs[base + e];
        sh_sn[warp][e] = sn[base + e];
        sh_b[warp][e] = col[base + 1 + e];
      }
      __syncwarp();
      if (lane == 0) {
        for (int e = 0; e < m; ++e) {
          const double c = sh_cs[warp][e], s = sh_sn[warp][e], b = sh_b[warp][e];
          col[base + e] = c * t + s * b;
          t = -s * t + c * b;
        }
      }
      __syncwarp();
    }
    if (lane != 0) continue;
    double c, s;
    givens_cs(t, hk1, c, s);
    cs[k] = c;
    sn[k] = s;
    col[k] = c * t + s * hk1;
    col[k + 1] = 0.0;
    const double gk = g[k];
    g[k + 1] = -s * gk;
    g[k] = c * gk;
    const double res = fabs(g[k + 1]);
    ws.hist[r * (ws.max_iter + 2) + k + 1] = res / q.bnorm;
    q.kconv = k + 1;
    int done = 0, flag = 0;
    if (!isfinite(res) || !isfinite(col[k])) {
      done = 1;
      flag = 4;
    } else if (res <= st->tol * q.bnorm) {
      done = 1;
      flag = 1;
    } else if (hk1 == 0.0) {
      done = 1;
      flag = 3;
    } else if (k + 1 >= st->max_iter) {
      done = 1;
      flag = 2;
    }
    q.done = done;
    q.flag = flag;
    if (!done) atomicAdd(&active, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st->k = k + 1;
    st->active = active;
    if (has_cond) cudaGraphSetConditional(cond, active > 0 ? 1u : 0u);
  }
}

void launch_givens(const KrylovWs &ws, cudaGraphConditionalHandle cond, int has_cond,
                   cudaStream_t s) {
  launch_pdl(kPdlKrylov, givens_kernel, dim3(1), dim3(ws.R == 1 ? 32 : 128), 0, s, ws, cond,
             has_cond);
  IGA_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ finish
// y_r = R_r^{-1} g_r (rotated upper-triangular H_r, kconv_r x kconv_r), one warp per rhs.
__global__ void backsolve_kernel(KrylovWs ws) {
  const int r = blockIdx.x;
  const int k = ws.rs[r].kconv;
  const int lane = threadIdx.x;
  double *y = ws.y + r * (ws.max_iter + 2);
  const double *g = ws.g + r * (ws.max_iter + 2);
  const double *H = ws.H + r * ws.hstride;
  const long long lh = ws.max_iter + 1;
  for (int j = lane; j < k; j += 32) y[j] = g[j];
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    double yi = 0.0;
    if (lane == 0) {
      yi = y[i] / H[lh * i + i];
      y[i] = yi;
    }
    yi = __shfl_sync(0xffffffffu, yi, 0);
    __syncwarp();
    for (int j = lane; j < i; j += 32) y[j] -= H[lh * i + j] * yi;
    __syncwarp();
  }
}

__device__ __forceinline__ double z_val(double v) { return v; }
// FP32 basis entries (precision form) widened on the integer units (fp_widen.h)
__device__ __forceinline__ double z_val(float v) { return widen_f32(v); }

template <class TZ>
__global__ void update_x_kernel(KrylovWs ws, const TZ *__restrict__ Z,
                                const double *__restrict__ x0, int use_x0,
                                double *__restrict__ x) {
  const int r = blockIdx.y;
  const int k = ws.rs[r].kconv;
  const double *y = ws.y + r * (ws.max_iter + 2);
  const double *x0r = x0 + (long long)r * ws.N;
  double *xr = x + (long long)r * ws.N;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ws.N;
       i += (long long)gridDim.x * blockDim.x) {
    double s = use_x0 ? x0r[i] : 0.0;
    for (int j = 0; j < k; ++j)
      s = fma(__ldg(y + j), z_val(Z[((long long)j * ws.R + r) * ws.N + i]), s);
    xr[i] = s;
  }
}

void launch_finish(const KrylovWs &ws, const double *x0, int use_x0, double *x, cudaStream_t s) {
  backsolve_kernel<<<ws.R, 32, 0, s>>>(ws);
  IGA_LAUNCH_CHECK();
  const dim3 grid(ws.nblk, ws.R);
  if (ws.z_fp32)
    update_x_kernel<float><<<grid, kRT, 0, s>>>(ws, (const float *)ws.Z, x0, use_x0, x);
  else
    update_x_kernel<double><<<grid, kRT, 0, s>>>(ws, (const double *)ws.Z, x0, use_x0, x);
  IGA_LAUNCH_CHECK();
}

// r = b - Ax; relres_true_r = ||r_r|| / ||b_r||
__global__ void __launch_bounds__(kRT) residual_kernel(KrylovWs ws, const double *__restrict__ b,
                                                       const double *__restrict__ Ax,
                                                       double *__restrict__ res) {
  __shared__ double red[kWarps][kJC];
  const int r = blockIdx.y;
  const long long o = (long long)r * ws.N;
  long long lo, hi;
  row_range(ws.N, lo, hi);
  double acc[kJC] = {};
  for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
    const double v = b[o + i] - Ax[o + i];
    res[o + i] = v;
    acc[0] = fma(v, v, acc[0]);
  }
  double *part = ws.partials + r * ws.pstride;
  block_store_partials(acc, 1, 0, part, gridDim.x, red);
  if (!arrive_last(ws.counter + r)) return;
  last_block_reduce(part, gridDim.x, 1, ws.scal + 8 * r + 3, 0, nullptr);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double bn = ws.rs[r].bnorm, rn = sqrt(ws.scal[8 * r + 3]);
    ws.rs[r].relres_true = bn > 0.0 ? rn / bn : rn;
    ws.counter[r] = 0;
  }
}

void launch_residual_norm(const KrylovWs &ws, const double *b, const double *Ax, double *r,
                          cudaStream_t s) {
  residual_kernel<<<dim3(ws.nblk, ws.R), kRT, 0, s>>>(ws, b, Ax, r);
  IGA_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ elementwise
__global__ void axpby_kernel(const double *__restrict__ x, const double *__restrict__ y, double a,
                             double b, double *__restrict__ out, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}

void launch_axpby(const double *x, const double *y, double a, double b, double *out, long long N,
                  cudaStream_t s) {
  const int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 8);
  axpby_kernel<<<blocks, 256, 0, s>>>(x, y, a, b, out, N);
  IGA_LAUNCH_CHECK();
}

void preload_kernels_krylov() {
  cudaFuncAttributes a;
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, init_norms_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, init_finalize_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, scale_v0_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, cgs_pass1_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, cgs_pass1_op_kernel<3>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, cgs_pass1_op_kernel<4>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, cgs_pass1_op_kernel<5>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, cgs_pass1_op_kernel<6>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, cgs_pass1_op_kernel<7>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, cgs_pass2_kernel));
  // the largest Krylov workspace's coefficients plus the stash (once per device, before any
  // capture: the attribute belongs to the kernel)
  IGA_CUDA_TRY(cudaFuncSetAttribute(cgs_pass2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)pass2_smem(kMaxIter, true)));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, cgs_pass3_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, givens_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, backsolve_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, update_x_kernel<double>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, update_x_kernel<float>));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, residual_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, axpby_kernel));
}

}  // namespace iga
