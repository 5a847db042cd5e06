// FP64 throughput probes: the ceiling that every FP64 kernel of the library is graded
// against.  Not part of the method; a measurement utility.
//
// GB300 executes FP64 on a narrow unit shared by FP64 FMAs and the FP64 tensor path
// (mma.sync .f64).  Two probes keep every SM sub-partition's FP64 unit busy:
//   kind 0  mma.sync m8n8k4 .f64: each warp keeps kChains independent accumulator
//           fragments and issues one MMA per fragment per loop turn (512 FLOP each);
//   kind 1  FP64 FMAs: each thread keeps kChains independent FMA chains (2 FLOP each);
//   kind 2  both: even warps run kind 0's loop, odd warps kind 1's;
//   kind 3  both: every warp runs kind 0's and kind 1's chains in one loop.
// Measured on GB300: kinds 2 and 3 reach 950-1034 GFLOP/s, no more than either path alone
// (mma.sync 1053-1098, FMA 1012-1243 in the same runs), so the two paths share one unit.
// The grid is sized to the SM count with kWarpsPerSm warps per SM (several per
// sub-partition), operands live in registers, and the result is stored (into a
// library-owned device array) only under a condition the compiler cannot prove false,
// so no work is eliminated.
#include "iga_internal.h"

namespace iga {

constexpr int kPeakChains = 8;
constexpr int kPeakWarpsPerSm = 16;
// external linkage: stores to it cannot be dropped as unobservable
__device__ double g_probe_sink[kPeakWarpsPerSm * 32];

__global__ void __launch_bounds__(kPeakWarpsPerSm * 32)
    fp64_dmma_probe_kernel(int reps, double seed) {
  double c[kPeakChains][2];
#pragma unroll
  for (int q = 0; q < kPeakChains; ++q) {
    c[q][0] = seed * (q + 1);
    c[q][1] = seed * (q + 2);
  }
  const double a = 1.0 + 1e-9 * threadIdx.x, b = 1.0 - 1e-9 * threadIdx.x;
  for (int r = 0; r < reps; ++r) {
#pragma unroll
    for (int q = 0; q < kPeakChains; ++q)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[q][0]), "+d"(c[q][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kPeakChains; ++q) s += c[q][0] + c[q][1];
  if (s == 12345.6789) g_probe_sink[threadIdx.x] = s;  // never true for the seeds used
}

// Both paths at once: MODE 2 splits the warps (even: mma.sync, odd: FMA), MODE 3 gives every
// warp both sets of chains.
template <int MODE>
__global__ void __launch_bounds__(kPeakWarpsPerSm * 32)
    fp64_mixed_probe_kernel(int reps, double seed) {
  double c[kPeakChains][2], f[kPeakChains];
#pragma unroll
  for (int q = 0; q < kPeakChains; ++q) {
    c[q][0] = seed * (q + 1);
    c[q][1] = seed * (q + 2);
    f[q] = seed * (q + 3);
  }
  const double a = 1.0 + 1e-9 * threadIdx.x, b = 1.0 - 1e-9 * threadIdx.x;
  const double fa = 1.0 - 1e-12 * threadIdx.x, fb = 1e-12 * blockIdx.x;
  const int warp = threadIdx.x >> 5;
  const bool do_mma = MODE == 3 || (warp & 1) == 0;  // warp-uniform
  const bool do_fma = MODE == 3 || (warp & 1) == 1;
  for (int r = 0; r < reps; ++r) {
    if (do_mma) {
#pragma unroll
      for (int q = 0; q < kPeakChains; ++q)
        asm volatile(
            "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
            : "+d"(c[q][0]), "+d"(c[q][1])
            : "d"(a), "d"(b));
    }
    if (do_fma) {
#pragma unroll
      for (int q = 0; q < kPeakChains; ++q) f[q] = fma(f[q], fa, fb);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kPeakChains; ++q) s += c[q][0] + c[q][1] + f[q];
  if (s == 12345.6789) g_probe_sink[threadIdx.x] = s;  // never true for the seeds used
}

__global__ void __launch_bounds__(kPeakWarpsPerSm * 32)
    fp64_fma_probe_kernel(int reps, double seed) {
  double c[kPeakChains];
#pragma unroll
  for (int q = 0; q < kPeakChains; ++q) c[q] = seed * (q + 1);
  const double a = 1.0 - 1e-12 * threadIdx.x, b = 1e-12 * blockIdx.x;
  for (int r = 0; r < reps; ++r) {
#pragma unroll
    for (int q = 0; q < kPeakChains; ++q) c[q] = fma(c[q], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kPeakChains; ++q) s += c[q];
  if (s == 12345.6789) g_probe_sink[threadIdx.x] = s;
}

}  // namespace iga

extern "C" iga_status iga_fp64_probe(int kind, int reps, void *stream, double *flops) {
  using namespace iga;
  try {
    if (kind < 0 || kind > 3) throw Error{IGA_ERR_INVALID_ARG, "kind must be 0, 1, 2 or 3"};
    if (reps < 1 || reps > (1 << 24)) throw Error{IGA_ERR_INVALID_ARG, "reps out of range"};
    int dev = 0, nsm = 0;
    IGA_CUDA_TRY(cudaGetDevice(&dev));
    IGA_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const dim3 grid(nsm), block(kPeakWarpsPerSm * 32);
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 0)
      fp64_dmma_probe_kernel<<<grid, block, 0, s>>>(reps, 0.5);
    else if (kind == 1)
      fp64_fma_probe_kernel<<<grid, block, 0, s>>>(reps, 0.5);
    else if (kind == 2)
      fp64_mixed_probe_kernel<2><<<grid, block, 0, s>>>(reps, 0.5);
    else
      fp64_mixed_probe_kernel<3><<<grid, block, 0, s>>>(reps, 0.5);
    IGA_LAUNCH_CHECK();
    const double warps = (double)nsm * kPeakWarpsPerSm;
    // per loop turn and chain: 512 FLOP per mma.sync warp, 64 per FMA warp
    const double mma_w = kind == 0 || kind == 3 ? warps : (kind == 2 ? warps / 2 : 0.0);
    const double fma_w = kind == 1 || kind == 3 ? warps : (kind == 2 ? warps / 2 : 0.0);
    const double per = mma_w * 512.0 + fma_w * 32.0 * 2.0;
    if (flops) *flops = per * kPeakChains * (double)reps;
    return IGA_OK;
  } catch (const Error &e) {
    set_error(e.msg);
    return e.status;
  } catch (const std::exception &e) {
    set_error(e.what());
    return IGA_ERR_CUDA;
  }
}
