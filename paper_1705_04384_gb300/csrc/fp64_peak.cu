// FP64 throughput probes: the ceiling that every FP64 kernel of the library is graded
// against.  Not part of the method; a measurement utility.
//
// GB300 executes FP64 on a narrow unit shared by FP64 FMAs and the FP64 tensor path
// (mma.sync .f64).  Two probes keep every SM sub-partition's FP64 unit busy:
//   kind 0  mma.sync m8n8k4 .f64: each warp keeps kChains independent accumulator
//           fragments and issues one MMA per fragment per loop turn (512 FLOP each);
//   kind 1  FP64 FMAs: each thread keeps kChains independent FMA chains (2 FLOP each).
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
    if (kind != 0 && kind != 1) throw Error{IGA_ERR_INVALID_ARG, "kind must be 0 or 1"};
    if (reps < 1 || reps > (1 << 24)) throw Error{IGA_ERR_INVALID_ARG, "reps out of range"};
    int dev = 0, nsm = 0;
    IGA_CUDA_TRY(cudaGetDevice(&dev));
    IGA_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const dim3 grid(nsm), block(kPeakWarpsPerSm * 32);
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 0)
      fp64_dmma_probe_kernel<<<grid, block, 0, s>>>(reps, 0.5);
    else
      fp64_fma_probe_kernel<<<grid, block, 0, s>>>(reps, 0.5);
    IGA_LAUNCH_CHECK();
    const double warps = (double)nsm * kPeakWarpsPerSm;
    const double per = kind == 0 ? warps * 512.0 : warps * 32.0 * 2.0;
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
