// BiCGStab kernels (van der Vorst 1992; the solver of Sec. 5), right preconditioned:
// the FD solve is applied to p and s, x is updated with M^{-1} p and M^{-1} s.  One
// right-hand side.  The vector updates, dot products and the scalar recurrences run
// in these kernels; the FD solves and the operator are the library's own launches.
// The iteration state lives in device memory (BicgState) so that one captured CUDA
// graph with a device-side while loop serves every iteration.
//
// Every reduction is a fixed partition of the rows into blocks, a fixed-order sum in
// each block and a fixed-order sum of the block partials by the last block to finish
// (atomic ticket, no spinning): results are bitwise reproducible.
//
// Stop test (the paper's half-iteration counting): after the BiCG half of iteration
// k (s = r - alpha v) and after the GMRES(1) half (r = s - omega t), on the
// recursively updated residual, ||.|| <= tol ||b||.  A solve that stops after the
// BiCG half takes x += alpha M^{-1} p only and reports 2k - 1 half steps.
#include <cmath>

#include "iga_internal.h"

namespace iga {

constexpr int kBT = 256, kBW = kBT / 32;

__device__ __forceinline__ double bwarp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void brow_range(long long N, long long &lo, long long &hi) {
  const long long chunk = (N + gridDim.x - 1) / gridDim.x;
  lo = (long long)blockIdx.x * chunk;
  hi = min(N, lo + chunk);
}

// Block sums of cnt <= 3 per-thread values -> partial[q * gridDim.x + blockIdx.x].
__device__ void bstore_partials(const double (&a)[3], int cnt, double *partial) {
  __shared__ double red[3][kBW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (q >= cnt) break;
    const double v = bwarp_sum(a[q]);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int w = 0; w < kBW; ++w) s += red[threadIdx.x][w];
    partial[(long long)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
  __syncthreads();
}

// True in exactly one block (the last to arrive), which then sees all partials.
__device__ bool barrive_last(unsigned int *counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// In the last block: out[q] = sum_b partial[q * nblk + b] in block order (warp q sums
// entry q); every thread of the block receives the sums.  A lane loads its partials
// (up to kBLdPer per round) before adding them in the same order, one L2 round trip per
// 32 kBLdPer partials instead of one per 32.
constexpr int kBLdPer = 10;
__device__ void bfinal_sums(const double *partial, int cnt, double (&out)[3]) {
  __shared__ double res[3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < cnt) {
    const double *pq = partial + (long long)warp * gridDim.x;
    const int nblk = (int)gridDim.x;
    double s = 0.0;
    for (int b0 = 0; b0 < nblk; b0 += 32 * kBLdPer) {
      double t[kBLdPer];
#pragma unroll
      for (int q = 0; q < kBLdPer; ++q) {
        const int b = b0 + lane + 32 * q;
        t[q] = b < nblk ? __ldcg(pq + b) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < kBLdPer; ++q) s += t[q];
    }
    s = bwarp_sum(s);
    if (lane == 0) res[warp] = s;
  }
  __syncthreads();
  for (int q = 0; q < 3; ++q) out[q] = q < cnt ? res[q] : 0.0;
  __syncthreads();
}

// ------------------------------------------------------------------ prologue
// r = r0, rhat = r0, p = v = 0, x = x0 (or 0); ||b||^2, ||r0||^2 -> state, hist[0].
__global__ void __launch_bounds__(kBT) bicg_init_kernel(BicgWs ws, const double *__restrict__ b,
                                                        const double *__restrict__ r0,
                                                        const double *__restrict__ x0,
                                                        cudaGraphConditionalHandle cond,
                                                        int has_cond) {
  long long lo, hi;
  brow_range(ws.N, lo, hi);
  double a[3] = {0.0, 0.0, 0.0};
  for (long long i = lo + threadIdx.x; i < hi; i += kBT) {
    const double bi = b[i], ri = r0[i];
    ws.r[i] = ri;
    ws.rhat[i] = ri;
    ws.p[i] = 0.0;
    ws.v[i] = 0.0;
    ws.x[i] = x0 ? x0[i] : 0.0;
    a[0] = fma(bi, bi, a[0]);
    a[1] = fma(ri, ri, a[1]);
  }
  bstore_partials(a, 2, ws.partials);
  if (!barrive_last(ws.counter)) return;
  double s[3];
  bfinal_sums(ws.partials, 2, s);
  if (threadIdx.x == 0) {
    BicgState &st = *ws.st;
    const double bn = sqrt(s[0]), rn = sqrt(s[1]);
    st.bnorm = bn;
    st.rho = s[1];  // (rhat, r0) with rhat = r0
    st.rho_prev = st.alpha = st.omega = 1.0;
    st.k = 1;
    st.steps = 0;
    st.half = 0;
    st.relres_true = 0.0;
    ws.hist[0] = bn > 0.0 ? rn / bn : 0.0;
    int done = 0, flag = 2;
    if (!isfinite(bn) || !isfinite(rn)) {
      done = 1;
      flag = 4;
    } else if (rn <= st.tol * bn) {
      done = 1;
      flag = 0;
    } else if (st.max_iter <= 0) {
      done = 1;
    }
    st.done = done;
    st.flag = flag;
    *ws.counter = 0;
    if (has_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
  }
}

// ------------------------------------------------------------------ iteration
// p = r + beta (p - omega v), beta = (rho / rho_prev)(alpha / omega)  (first: p = r)
__global__ void bicg_p_kernel(BicgWs ws) {
  const BicgState &st = *ws.st;
  if (st.done) return;
  const double beta = (st.rho / st.rho_prev) * (st.alpha / st.omega), om = st.omega;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ws.N;
       i += (long long)gridDim.x * blockDim.x)
    ws.p[i] = fma(beta, ws.p[i] - om * ws.v[i], ws.r[i]);
}

// alpha = rho / (rhat, v)
__global__ void __launch_bounds__(kBT) bicg_alpha_kernel(BicgWs ws) {
  if (ws.st->done) return;
  long long lo, hi;
  brow_range(ws.N, lo, hi);
  double a[3] = {0.0, 0.0, 0.0};
  for (long long i = lo + threadIdx.x; i < hi; i += kBT) a[0] = fma(ws.rhat[i], ws.v[i], a[0]);
  bstore_partials(a, 1, ws.partials);
  if (!barrive_last(ws.counter)) return;
  double s[3];
  bfinal_sums(ws.partials, 1, s);
  if (threadIdx.x == 0) {
    BicgState &st = *ws.st;
    if (!isfinite(s[0])) {
      st.done = 1;
      st.flag = 4;
    } else if (s[0] == 0.0) {
      st.done = 1;
      st.flag = 3;
    } else {
      st.alpha = st.rho / s[0];
    }
    *ws.counter = 0;
  }
}

// s = r - alpha v; ||s|| -> hist[2k - 1]; half-step stop test
__global__ void __launch_bounds__(kBT) bicg_s_kernel(BicgWs ws) {
  if (ws.st->done) return;
  const double alpha = ws.st->alpha;
  long long lo, hi;
  brow_range(ws.N, lo, hi);
  double a[3] = {0.0, 0.0, 0.0};
  for (long long i = lo + threadIdx.x; i < hi; i += kBT) {
    const double si = fma(-alpha, ws.v[i], ws.r[i]);
    ws.s[i] = si;
    a[0] = fma(si, si, a[0]);
  }
  bstore_partials(a, 1, ws.partials);
  if (!barrive_last(ws.counter)) return;
  double s[3];
  bfinal_sums(ws.partials, 1, s);
  if (threadIdx.x == 0) {
    BicgState &st = *ws.st;
    const double sn = sqrt(s[0]);
    ws.hist[2 * st.k - 1] = st.bnorm > 0.0 ? sn / st.bnorm : 0.0;
    st.steps = 2 * st.k - 1;
    if (!isfinite(sn)) {
      st.done = 1;
      st.flag = 4;
    } else if (sn <= st.tol * st.bnorm) {
      st.half = 1;  // x takes alpha M^-1 p only; the solve ends after the update
    }
    *ws.counter = 0;
  }
}

// omega = (t, s) / (t, t)
__global__ void __launch_bounds__(kBT) bicg_omega_kernel(BicgWs ws) {
  if (ws.st->done || ws.st->half) return;
  long long lo, hi;
  brow_range(ws.N, lo, hi);
  double a[3] = {0.0, 0.0, 0.0};
  for (long long i = lo + threadIdx.x; i < hi; i += kBT) {
    const double ti = ws.t[i];
    a[0] = fma(ti, ws.s[i], a[0]);
    a[1] = fma(ti, ti, a[1]);
  }
  bstore_partials(a, 2, ws.partials);
  if (!barrive_last(ws.counter)) return;
  double s[3];
  bfinal_sums(ws.partials, 2, s);
  if (threadIdx.x == 0) {
    BicgState &st = *ws.st;
    if (!isfinite(s[0]) || !isfinite(s[1])) {
      st.done = 1;
      st.flag = 4;
    } else if (s[1] == 0.0) {
      st.done = 1;
      st.flag = 3;
    } else {
      st.omega = s[0] / s[1];
    }
    *ws.counter = 0;
  }
}

// x += alpha phat (+ omega shat); r = s - omega t; ||r||, (rhat, r); full-step stop test,
// next rho, loop condition
__global__ void __launch_bounds__(kBT) bicg_xr_kernel(BicgWs ws, cudaGraphConditionalHandle cond,
                                                      int has_cond) {
  const BicgState &cst = *ws.st;
  if (cst.done) return;
  const int half = cst.half;
  const double alpha = cst.alpha, omega = cst.omega;
  long long lo, hi;
  brow_range(ws.N, lo, hi);
  double a[3] = {0.0, 0.0, 0.0};
  for (long long i = lo + threadIdx.x; i < hi; i += kBT) {
    if (half) {
      ws.x[i] = fma(alpha, ws.phat[i], ws.x[i]);
    } else {
      ws.x[i] = fma(omega, ws.shat[i], fma(alpha, ws.phat[i], ws.x[i]));
      const double ri = fma(-omega, ws.t[i], ws.s[i]);
      ws.r[i] = ri;
      a[0] = fma(ri, ri, a[0]);
      a[1] = fma(ws.rhat[i], ri, a[1]);
    }
  }
  bstore_partials(a, 2, ws.partials);
  if (!barrive_last(ws.counter)) return;
  double s[3];
  bfinal_sums(ws.partials, 2, s);
  if (threadIdx.x == 0) {
    BicgState &st = *ws.st;
    if (half) {
      st.done = 1;
      st.flag = 0;
    } else {
      const double rn = sqrt(s[0]);
      ws.hist[2 * st.k] = st.bnorm > 0.0 ? rn / st.bnorm : 0.0;
      st.steps = 2 * st.k;
      if (!isfinite(rn) || !isfinite(s[1])) {
        st.done = 1;
        st.flag = 4;
      } else if (rn <= st.tol * st.bnorm) {
        st.done = 1;
        st.flag = 0;
      } else {
        st.rho_prev = st.rho;
        st.rho = s[1];
        if (st.rho == 0.0 || st.omega == 0.0) {
          st.done = 1;
          st.flag = 3;
        } else if (st.k >= st.max_iter) {
          st.done = 1;
          st.flag = 2;
        } else {
          st.k += 1;
        }
      }
    }
    *ws.counter = 0;
    if (has_cond) cudaGraphSetConditional(cond, st.done ? 0u : 1u);
  }
}

// ------------------------------------------------------------------ epilogue
// relres_true = ||b - Ax|| / ||b||
__global__ void __launch_bounds__(kBT) bicg_residual_kernel(BicgWs ws, const double *__restrict__ b,
                                                            const double *__restrict__ Ax) {
  long long lo, hi;
  brow_range(ws.N, lo, hi);
  double a[3] = {0.0, 0.0, 0.0};
  for (long long i = lo + threadIdx.x; i < hi; i += kBT) {
    const double ri = b[i] - Ax[i];
    a[0] = fma(ri, ri, a[0]);
  }
  bstore_partials(a, 1, ws.partials);
  if (!barrive_last(ws.counter)) return;
  double s[3];
  bfinal_sums(ws.partials, 1, s);
  if (threadIdx.x == 0) {
    BicgState &st = *ws.st;
    st.relres_true = st.bnorm > 0.0 ? sqrt(s[0]) / st.bnorm : 0.0;
    *ws.counter = 0;
  }
}

// ------------------------------------------------------------------ launches
static int ew_blocks(long long N) {
  return (int)std::min<long long>((N + kBT - 1) / kBT, 152LL * 8);
}

void launch_bicg_init(const BicgWs &ws, const double *b, const double *r0, const double *x0,
                      cudaGraphConditionalHandle cond, int has_cond, cudaStream_t s) {
  bicg_init_kernel<<<ws.nblk, kBT, 0, s>>>(ws, b, r0, x0, cond, has_cond);
  IGA_LAUNCH_CHECK();
}
void launch_bicg_p(const BicgWs &ws, cudaStream_t s) {
  bicg_p_kernel<<<ew_blocks(ws.N), kBT, 0, s>>>(ws);
  IGA_LAUNCH_CHECK();
}
void launch_bicg_alpha(const BicgWs &ws, cudaStream_t s) {
  bicg_alpha_kernel<<<ws.nblk, kBT, 0, s>>>(ws);
  IGA_LAUNCH_CHECK();
}
void launch_bicg_s(const BicgWs &ws, cudaStream_t s) {
  bicg_s_kernel<<<ws.nblk, kBT, 0, s>>>(ws);
  IGA_LAUNCH_CHECK();
}
void launch_bicg_omega(const BicgWs &ws, cudaStream_t s) {
  bicg_omega_kernel<<<ws.nblk, kBT, 0, s>>>(ws);
  IGA_LAUNCH_CHECK();
}
void launch_bicg_xr(const BicgWs &ws, cudaGraphConditionalHandle cond, int has_cond,
                    cudaStream_t s) {
  bicg_xr_kernel<<<ws.nblk, kBT, 0, s>>>(ws, cond, has_cond);
  IGA_LAUNCH_CHECK();
}
void launch_bicg_residual(const BicgWs &ws, const double *b, const double *Ax, cudaStream_t s) {
  bicg_residual_kernel<<<ws.nblk, kBT, 0, s>>>(ws, b, Ax);
  IGA_LAUNCH_CHECK();
}

void preload_kernels_bicgstab() {
  cudaFuncAttributes a;
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, bicg_init_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, bicg_p_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, bicg_alpha_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, bicg_s_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, bicg_omega_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, bicg_xr_kernel));
  IGA_CUDA_TRY(cudaFuncGetAttributes(&a, bicg_residual_kernel));
}

}  // namespace iga
