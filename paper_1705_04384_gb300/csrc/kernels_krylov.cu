// GMRES kernels: deterministic reductions, classical Gram-Schmidt with one
// re-orthogonalization (CGS2) as batched GEMV passes with fused norms, Givens
// rotations of the Hessenberg column, back substitution and the solution update.
//
// The Krylov method is GMRES (Saad & Schultz, named in Sec. 3 of the paper); the
// Arnoldi step number k lives in device memory (SolveState::k) so that one CUDA
// graph replays every iteration.  Reductions over blocks are done by the last
// block to finish (atomic ticket, no spinning), always in block order, so results
// are bitwise reproducible and independent of scheduling.
#include <cmath>

#include "iga_internal.h"

namespace iga {

constexpr int kRT = 256;       // threads per reduction block
constexpr int kWarps = kRT / 32;
constexpr int kJC = 8;         // vectors per register chunk

int reduce_blocks(long long N) {
  long long b = (N + 2047) / 2048;
  if (b < 1) b = 1;
  if (b > 304) b = 304;
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

// Block-reduce acc[0..cnt) (cnt <= kJC) and store partial[(j0+q)*nblk + blockIdx.x].
__device__ __forceinline__ void block_store_partials(double (&acc)[kJC], int cnt, int j0,
                                                     double *partial, int nblk,
                                                     double (*red)[kJC]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kJC; ++q) acc[q] = warp_sum(acc[q]);
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < kJC; ++q) red[warp][q] = acc[q];
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
    partial[(long long)(j0 + threadIdx.x) * nblk + blockIdx.x] = s;
  }
  __syncthreads();
}

// Returns true in exactly one block (the last to arrive); that block then sees
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

// Sum partial[j*nblk + b] over b for j < cnt into out[j*ostride] (op: 0 store, 1 add).
__device__ void last_block_reduce(const double *partial, int nblk, int cnt, double *out,
                                  int op, double *out2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < cnt; j += kWarps) {
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += __ldcg(partial + (long long)j * nblk + b);
    s = warp_sum(s);
    if (lane == 0) {
      if (op == 0) out[j] = s; else out[j] += s;
      if (out2) out2[j] = s;
    }
  }
}

// ------------------------------------------------------------------ generic dot
__global__ void __launch_bounds__(kRT) dot_kernel(const double *__restrict__ x,
                                                  const double *__restrict__ y, long long N,
                                                  double *partial, unsigned int *counter,
                                                  double *out) {
  __shared__ double red[kWarps][kJC];
  long long lo, hi;
  row_range(N, lo, hi);
  double acc[kJC] = {};
  for (long long i = lo + threadIdx.x; i < hi; i += kRT) acc[0] = fma(x[i], y[i], acc[0]);
  block_store_partials(acc, 1, 0, partial, gridDim.x, red);
  if (!arrive_last(counter)) return;
  last_block_reduce(partial, gridDim.x, 1, out, 0, nullptr);
  if (threadIdx.x == 0) *counter = 0;
}

void launch_dot(const double *x, const double *y, long long N, const KrylovWs &ws, double *out,
                cudaStream_t s) {
  dot_kernel<<<ws.nblk, kRT, 0, s>>>(x, y, N, ws.partials, ws.counter, out);
  IGA_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ init
// scal[0] = ||b||^2, scal[1] = ||r0||^2 computed before this kernel.
__global__ void init_finalize_kernel(KrylovWs ws, cudaGraphConditionalHandle cond, int has_cond) {
  SolveState *st = ws.st;
  const double bn = sqrt(ws.scal[0]);
  const double beta = sqrt(ws.scal[1]);
  st->bnorm = bn;
  st->beta = beta;
  st->k = 0;
  st->relres_true = 0.0;
  ws.g[0] = beta;
  ws.hist[0] = bn > 0.0 ? beta / bn : 0.0;
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
  st->done = done;
  st->flag = flag;
  if (has_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
}

__global__ void scale_v0_kernel(KrylovWs ws, const double *__restrict__ r) {
  const double beta = ws.st->beta;
  const int ok = ws.st->done == 0;
  const double inv = ok ? 1.0 / beta : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ws.N;
       i += (long long)gridDim.x * blockDim.x)
    ws.V[i] = r[i] * inv;
}

void launch_init_solve(const KrylovWs &ws, const double *r, cudaGraphConditionalHandle cond,
                       int has_cond, cudaStream_t s) {
  init_finalize_kernel<<<1, 1, 0, s>>>(ws, cond, has_cond);
  IGA_LAUNCH_CHECK();
  scale_v0_kernel<<<ws.nblk, kRT, 0, s>>>(ws, r);
  IGA_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ CGS2
// pass 1: h1 = V_{0..k}^T w  -> H[0..k, k]
__global__ void __launch_bounds__(kRT) cgs_pass1_kernel(KrylovWs ws, const double *__restrict__ w) {
  __shared__ double red[kWarps][kJC];
  const int k = ws.st->k;
  const int nv = k + 1;
  const long long ldh = ws.max_iter + 1;
  long long lo, hi;
  row_range(ws.N, lo, hi);
  for (int j0 = 0; j0 < nv; j0 += kJC) {
    const int cnt = min(kJC, nv - j0);
    double acc[kJC] = {};
    for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
      const double wv = w[i];
#pragma unroll
      for (int q = 0; q < kJC; ++q)
        if (q < cnt) acc[q] = fma(ws.V[(long long)(j0 + q) * ws.ldv + i], wv, acc[q]);
    }
    block_store_partials(acc, cnt, j0, ws.partials, gridDim.x, red);
  }
  if (!arrive_last(ws.counter)) return;
  last_block_reduce(ws.partials, gridDim.x, nv, ws.H + ldh * k, 0, nullptr);
  if (threadIdx.x == 0) *ws.counter = 0;
}

// pass 2: w -= V h1; h2 = V^T w -> H[0..k,k] += h2, y = h2
__global__ void __launch_bounds__(kRT) cgs_pass2_kernel(KrylovWs ws, double *__restrict__ w) {
  __shared__ double red[kWarps][kJC];
  const int k = ws.st->k;
  const int nv = k + 1;
  const long long ldh = ws.max_iter + 1;
  const double *h1 = ws.H + ldh * k;
  long long lo, hi;
  row_range(ws.N, lo, hi);
  for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
    double s = 0.0;
    for (int j = 0; j < nv; ++j) s = fma(ws.V[(long long)j * ws.ldv + i], __ldg(h1 + j), s);
    w[i] -= s;
  }
  for (int j0 = 0; j0 < nv; j0 += kJC) {
    const int cnt = min(kJC, nv - j0);
    double acc[kJC] = {};
    for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
      const double wv = w[i];
#pragma unroll
      for (int q = 0; q < kJC; ++q)
        if (q < cnt) acc[q] = fma(ws.V[(long long)(j0 + q) * ws.ldv + i], wv, acc[q]);
    }
    block_store_partials(acc, cnt, j0, ws.partials, gridDim.x, red);
  }
  if (!arrive_last(ws.counter)) return;
  last_block_reduce(ws.partials, gridDim.x, nv, ws.H + ldh * k, 1, ws.y);
  if (threadIdx.x == 0) *ws.counter = 0;
}

// pass 3: w -= V h2; H[k+1,k] = ||w||
__global__ void __launch_bounds__(kRT) cgs_pass3_kernel(KrylovWs ws, double *__restrict__ w) {
  __shared__ double red[kWarps][kJC];
  const int k = ws.st->k;
  const int nv = k + 1;
  const long long ldh = ws.max_iter + 1;
  long long lo, hi;
  row_range(ws.N, lo, hi);
  double acc[kJC] = {};
  for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
    double s = 0.0;
    for (int j = 0; j < nv; ++j) s = fma(ws.V[(long long)j * ws.ldv + i], __ldg(ws.y + j), s);
    const double v = w[i] - s;
    w[i] = v;
    acc[0] = fma(v, v, acc[0]);
  }
  block_store_partials(acc, 1, 0, ws.partials, gridDim.x, red);
  if (!arrive_last(ws.counter)) return;
  last_block_reduce(ws.partials, gridDim.x, 1, ws.scal + 2, 0, nullptr);
  __syncthreads();
  if (threadIdx.x == 0) {
    ws.H[ldh * k + k + 1] = sqrt(ws.scal[2]);
    *ws.counter = 0;
  }
}

// v_{k+1} = w / H[k+1,k]
__global__ void normalize_kernel(KrylovWs ws, const double *__restrict__ w) {
  const int k = ws.st->k;
  const long long ldh = ws.max_iter + 1;
  const double h = ws.H[ldh * k + k + 1];
  const double inv = h > 0.0 ? 1.0 / h : 0.0;
  double *v = ws.V + (long long)(k + 1) * ws.ldv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ws.N;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = w[i] * inv;
}

void launch_cgs2(const KrylovWs &ws, double *w, cudaStream_t s) {
  cgs_pass1_kernel<<<ws.nblk, kRT, 0, s>>>(ws, w);
  IGA_LAUNCH_CHECK();
  cgs_pass2_kernel<<<ws.nblk, kRT, 0, s>>>(ws, w);
  IGA_LAUNCH_CHECK();
  cgs_pass3_kernel<<<ws.nblk, kRT, 0, s>>>(ws, w);
  IGA_LAUNCH_CHECK();
  normalize_kernel<<<ws.nblk, kRT, 0, s>>>(ws, w);
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

// Rotate column k of H by the previous rotations, build rotation k, update g and
// the residual estimate, advance k and decide whether to continue.
__global__ void givens_kernel(KrylovWs ws, cudaGraphConditionalHandle cond, int has_cond) {
  SolveState *st = ws.st;
  const int k = st->k;
  const long long ldh = ws.max_iter + 1;
  double *col = ws.H + ldh * k;
  const double hk1 = col[k + 1];
  for (int i = 0; i < k; ++i) {
    const double a = col[i], b = col[i + 1];
    col[i] = ws.cs[i] * a + ws.sn[i] * b;
    col[i + 1] = -ws.sn[i] * a + ws.cs[i] * b;
  }
  double c, s;
  givens_cs(col[k], col[k + 1], c, s);
  ws.cs[k] = c;
  ws.sn[k] = s;
  col[k] = c * col[k] + s * col[k + 1];
  col[k + 1] = 0.0;
  const double gk = ws.g[k];
  ws.g[k + 1] = -s * gk;
  ws.g[k] = c * gk;
  const double res = fabs(ws.g[k + 1]);
  ws.hist[k + 1] = res / st->bnorm;
  st->k = k + 1;
  int done = 0, flag = 0;
  if (!isfinite(res) || !isfinite(col[k])) {
    done = 1;
    flag = 4;
  } else if (res <= st->tol * st->bnorm) {
    done = 1;
    flag = 1;
  } else if (hk1 == 0.0) {
    done = 1;
    flag = 3;
  } else if (k + 1 >= st->max_iter) {
    done = 1;
    flag = 2;
  }
  st->done = done;
  st->flag = flag;
  if (has_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
}

void launch_givens(const KrylovWs &ws, cudaGraphConditionalHandle cond, int has_cond,
                   cudaStream_t s) {
  givens_kernel<<<1, 1, 0, s>>>(ws, cond, has_cond);
  IGA_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ finish
// y = R^{-1} g (R = rotated upper-triangular H, k x k), one warp.
__global__ void backsolve_kernel(KrylovWs ws) {
  const int k = ws.st->k;
  const long long ldh = ws.max_iter + 1;
  const int lane = threadIdx.x;
  for (int j = lane; j < k; j += 32) ws.y[j] = ws.g[j];
  __syncwarp();
  for (int i = k - 1; i >= 0; --i) {
    double yi = 0.0;
    if (lane == 0) {
      yi = ws.y[i] / ws.H[ldh * i + i];
      ws.y[i] = yi;
    }
    yi = __shfl_sync(0xffffffffu, yi, 0);
    __syncwarp();
    for (int j = lane; j < i; j += 32) ws.y[j] -= ws.H[ldh * i + j] * yi;
    __syncwarp();
  }
}

template <class TZ>
__global__ void update_x_kernel(KrylovWs ws, const TZ *__restrict__ Z, const double *__restrict__ x0,
                                int use_x0, double *__restrict__ x) {
  const int k = ws.st->k;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ws.N;
       i += (long long)gridDim.x * blockDim.x) {
    double s = use_x0 ? x0[i] : 0.0;
    for (int j = 0; j < k; ++j) s = fma(__ldg(ws.y + j), (double)Z[(long long)j * ws.ldz + i], s);
    x[i] = s;
  }
}

void launch_finish(const KrylovWs &ws, const double *x0, int use_x0, double *x, cudaStream_t s) {
  backsolve_kernel<<<1, 32, 0, s>>>(ws);
  IGA_LAUNCH_CHECK();
  if (ws.z_fp32)
    update_x_kernel<float><<<ws.nblk, kRT, 0, s>>>(ws, (const float *)ws.Z, x0, use_x0, x);
  else
    update_x_kernel<double><<<ws.nblk, kRT, 0, s>>>(ws, (const double *)ws.Z, x0, use_x0, x);
  IGA_LAUNCH_CHECK();
}

// r = b - Ax; relres_true = ||r|| / ||b||
__global__ void __launch_bounds__(kRT) residual_kernel(KrylovWs ws, const double *__restrict__ b,
                                                       const double *__restrict__ Ax,
                                                       double *__restrict__ r) {
  __shared__ double red[kWarps][kJC];
  long long lo, hi;
  row_range(ws.N, lo, hi);
  double acc[kJC] = {};
  for (long long i = lo + threadIdx.x; i < hi; i += kRT) {
    const double v = b[i] - Ax[i];
    r[i] = v;
    acc[0] = fma(v, v, acc[0]);
  }
  block_store_partials(acc, 1, 0, ws.partials, gridDim.x, red);
  if (!arrive_last(ws.counter)) return;
  last_block_reduce(ws.partials, gridDim.x, 1, ws.scal + 3, 0, nullptr);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double bn = ws.st->bnorm;
    ws.st->relres_true = bn > 0.0 ? sqrt(ws.scal[3]) / bn : sqrt(ws.scal[3]);
    *ws.counter = 0;
  }
}

void launch_residual_norm(const KrylovWs &ws, const double *b, const double *Ax, double *r,
                          cudaStream_t s) {
  residual_kernel<<<ws.nblk, kRT, 0, s>>>(ws, b, Ax, r);
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

__global__ void convert_f32_kernel(const float *__restrict__ x, double *__restrict__ out,
                                   long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)x[i];
}

void launch_convert_f32(const float *x, double *out, long long N, cudaStream_t s) {
  const int blocks = (int)std::min<long long>((N + 255) / 256, 152LL * 8);
  convert_f32_kernel<<<blocks, 256, 0, s>>>(x, out, N);
  IGA_LAUNCH_CHECK();
}

}  // namespace iga
