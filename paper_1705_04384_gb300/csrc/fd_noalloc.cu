// FD solve (eq. FD2D / FD3D) that allocates nothing: the two intermediate tensors
// of the mode-product chain live in a fixed, file-scope device array instead of
// memory obtained from cudaMalloc.
//
// Who needs it: callers that must not allocate device memory at the point where
// they apply the preconditioner -- code running under a fixed memory budget
// reserved up front, allocator-free real-time loops, or hosts whose own allocator
// owns all device memory and forbids other cudaMalloc calls.  They pass the FD
// factors, the input and the output; the library supplies only the scratch.
#include <mutex>

#include "iga_internal.h"

namespace iga {

// Scratch capacity: two tensors of up to kNoAllocMaxN doubles (2 x 16 MiB).  Every
// GPU on which this entry point runs keeps the array until the process exits.
constexpr long long kNoAllocMaxN = 1LL << 21;
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxN];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {};

// The array's name in host code is only a host-side stand-in: its device address
// is looked up once per device, with that device current.
double *noalloc_scratch() {
  int dev = 0;
  IGA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw Error{IGA_ERR_INVALID_ARG, "device index out of range"};
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      throw Error{IGA_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
    g_noalloc_ptr[dev] = static_cast<double *>(p);
  }
  return g_noalloc_ptr[dev];
}
}  // namespace

}  // namespace iga

extern "C" iga_status iga_precond_apply_noalloc(int d, int n, const double *Vt_dev,
                                                const double *U_dev, const double *lam_dev,
                                                const double *b_dev, double *s_dev,
                                                void *stream) {
  using namespace iga;
  try {
    if (d != 2 && d != 3) throw Error{IGA_ERR_INVALID_ARG, "d must be 2 or 3"};
    if (n < 1) throw Error{IGA_ERR_INVALID_ARG, "n must be positive"};
    if (!Vt_dev || !U_dev || !lam_dev || !b_dev || !s_dev)
      throw Error{IGA_ERR_INVALID_ARG, "null argument"};
    long long N = 1;
    for (int l = 0; l < d; ++l) N *= n;
    if (N > kNoAllocMaxN)
      throw Error{IGA_ERR_INVALID_ARG,
                  "N = n^d = " + std::to_string(N) +
                      " exceeds the 2097152-value static scratch of iga_precond_apply_noalloc"};
    cudaStream_t s = (cudaStream_t)stream;
    double *t0 = noalloc_scratch();
    double *t1 = t0 + kNoAllocMaxN;
    // Every entry of t0 / t1 is written before it is read, so nothing needs clearing.
    const int M = (int)(N / n);
    auto P = [](double *p) { return plain_ptr<double>(p); };
    auto Pc = [](const double *p) { return plain_ptr<const double>(p); };
    if (d == 2) {
      const FdScale sc{lam_dev, nullptr, lam_dev, n};
      launch_gemm_fp64<double>(Pc(b_dev), Vt_dev, P(t0), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t0), Vt_dev, P(t1), M, n, n, &sc, s);
      launch_gemm_fp64<double>(Pc(t1), U_dev, P(t0), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t0), U_dev, P(s_dev), M, n, n, nullptr, s);
    } else {
      const FdScale sc{lam_dev, lam_dev, lam_dev, n};
      launch_gemm_fp64<double>(Pc(b_dev), Vt_dev, P(t0), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t0), Vt_dev, P(t1), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t1), Vt_dev, P(t0), M, n, n, &sc, s);
      launch_gemm_fp64<double>(Pc(t0), U_dev, P(t1), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t1), U_dev, P(t0), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t0), U_dev, P(s_dev), M, n, n, nullptr, s);
    }
    return IGA_OK;
  } catch (const Error &e) {
    set_error(e.msg);
    return e.status;
  } catch (const std::exception &e) {
    set_error(e.what());
    return IGA_ERR_CUDA;
  }
}
