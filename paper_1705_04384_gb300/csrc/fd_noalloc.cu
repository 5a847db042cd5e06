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

// Scratch capacity: two tensors of up to kNoAllocMaxN doubles (2 x 16 MiB).  The array is
// reserved on a device when this file's module is loaded there -- with CUDA's default lazy
// loading, at the first call on that device; with CUDA_MODULE_LOADING=EAGER, on every
// device the library initialises -- and stays reserved until the process exits.
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
    // N = n^d, checked after every factor so that no product can wrap around
    long long N = 1;
    for (int l = 0; l < d; ++l) {
      if (n > kNoAllocMaxN || N * n > kNoAllocMaxN)
        throw Error{IGA_ERR_INVALID_ARG,
                    "N = n^d with n = " + std::to_string(n) + ", d = " + std::to_string(d) +
                        " exceeds the 2097152-value static scratch of iga_precond_apply_noalloc"};
      N *= n;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *t0 = noalloc_scratch();
    double *t1 = t0 + kNoAllocMaxN;
    // Every entry of t0 / t1 is written before it is read, so nothing needs clearing.
    const int M = (int)(N / n);
    const size_t nn = (size_t)n * n;
    // direction l's factors: V_l^T and U_l at l n^2, its eigenvalues at l n
    const double *Vt[3], *U[3], *lam[3];
    for (int l = 0; l < d; ++l) {
      Vt[l] = Vt_dev + l * nn;
      U[l] = U_dev + l * nn;
      lam[l] = lam_dev + (size_t)l * n;
    }
    auto P = [](double *p) { return plain_ptr<double>(p); };
    auto Pc = [](const double *p) { return plain_ptr<const double>(p); };
    // The g-th forward product contracts direction g with V_g^T, the g-th inverse product
    // with U_g (layout rotation: the contracted index is always the fastest); the diagonal
    // 1 / (lambda_{0,k1} + lambda_{1,k2} (+ lambda_{2,k3})) is fused into the d-th forward
    // product, whose rows are (k1, k2) in 3D (k1 in 2D) and whose columns are k_d.
    if (d == 2) {
      const FdScale sc{lam[0], nullptr, lam[1], n};
      launch_gemm_fp64<double>(Pc(b_dev), Vt[0], P(t0), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t0), Vt[1], P(t1), M, n, n, &sc, s);
      launch_gemm_fp64<double>(Pc(t1), U[0], P(t0), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t0), U[1], P(s_dev), M, n, n, nullptr, s);
    } else {
      const FdScale sc{lam[0], lam[1], lam[2], n};
      launch_gemm_fp64<double>(Pc(b_dev), Vt[0], P(t0), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t0), Vt[1], P(t1), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t1), Vt[2], P(t0), M, n, n, &sc, s);
      launch_gemm_fp64<double>(Pc(t0), U[0], P(t1), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t1), U[1], P(t0), M, n, n, nullptr, s);
      launch_gemm_fp64<double>(Pc(t0), U[2], P(s_dev), M, n, n, nullptr, s);
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
