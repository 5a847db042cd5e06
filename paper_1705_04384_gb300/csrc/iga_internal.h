// Internal declarations shared by the host setup, the CUDA kernels and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstddef>
#include <cstdint>
#include <memory>
#include <mutex>
#include <shared_mutex>
#include <string>
#include <vector>

#include "../../include/iga_fd.h"
#include "device_lock.h"

namespace iga {

constexpr int kMaxDim = 3;
constexpr int kMaxDeg = 6;
constexpr int kMaxBand = kMaxDeg + 1;
constexpr int kMaxIter = 4096;

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
struct Error {
  iga_status status;
  std::string msg;
};
#define IGA_CUDA_TRY(expr)                                                          \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess)                                                          \
      throw ::iga::Error{IGA_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
// Every kernel launch of the library is followed by IGA_LAUNCH_CHECK(), which also
// counts launches on the calling thread (used to report launches per solve).
extern thread_local long long g_launch_count;
#define IGA_LAUNCH_CHECK()                \
  do {                                    \
    ++::iga::g_launch_count;              \
    IGA_CUDA_TRY(cudaGetLastError());     \
  } while (0)

// ---------------------------------------------------------------- dependent launch
// Programmatic dependent launch: a kernel launched with it may be scheduled as soon as
// every block of the previous kernel in the stream has triggered; it waits
// (griddepcontrol.wait) for the previous kernel to complete and its writes to be visible
// before it touches global memory, and then triggers its own successor.
// In a captured graph the edges become programmatic edges.  Every per-iteration kernel
// calls pdl_entry() first (a no-op when it was launched without the attribute);
// launch_pdl is followed by IGA_LAUNCH_CHECK() like <<<>>>.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_entry() {
  // wait first: a kernel lets its successor start only once it runs itself, so at most one
  // kernel waits ahead (triggering before the wait let successive launches cascade and
  // settle unevenly on the SMs: back-to-back FD applies ran 2x slower)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;");
}
#endif

// Kernel groups that may use it; which ones do is a measured choice (pdl_mask(),
// overridable with the IGA_PDL environment variable, a bit mask of these groups).
enum PdlGroup : int { kPdlFd64 = 1, kPdlOperator = 2, kPdlKrylov = 4, kPdlTensorCore = 8 };
int pdl_mask();

template <class... KArgs, class... Args>
inline void launch_pdl(int group, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = (pdl_mask() & group) ? 1 : 0;
  IGA_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
}

// ---------------------------------------------------------------- index division
// Division by an invariant 32-bit divisor d >= 1 for dividends x < 2^31, by one high
// multiply, an add and a shift (Granlund & Montgomery, "Division by invariant integers
// using multiplication", 1994): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// x / d = (umulhi(x, m) + x) >> l.  The per-element index arithmetic of the operator
// passes uses it: a 64-bit integer division is a long instruction sequence that on
// GB300 also occupies the (slow) FP64 unit.
struct FastDiv {
  unsigned d, m;
  int l;
};
inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f{d, 1u, 0};
  while ((1ull << f.l) < d) ++f.l;
  f.m = (unsigned)(((1ull << 32) * ((1ull << f.l) - d)) / d + 1);
  return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ unsigned fdiv(unsigned x, const FastDiv &f) {
  return (__umulhi(x, f.m) + x) >> f.l;
}
#endif
// Element counts that the operator and pack kernels index with 32-bit arithmetic.
constexpr long long kMaxIndex32 = (1LL << 31) - 1;

// ---------------------------------------------------------------- device memory
template <class T> struct DevBuf {
  T *ptr = nullptr;
  size_t count = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    count = 0;
  }
  void alloc(size_t n) {
    if (n <= count && ptr) return;
    release();
    if (n == 0) return;
    cudaError_t e = cudaMalloc(&ptr, n * sizeof(T));
    if (e != cudaSuccess) {
      ptr = nullptr;
      (void)cudaGetLastError();
      throw Error{IGA_ERR_OOM, "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed"};
    }
    count = n;
  }
};

// A pointer whose element offset is read on the device from an iteration counter:
// base + (idx ? (*idx + off) : 0) * stride.  Lets one captured CUDA graph serve
// every Arnoldi step (the step number lives in device memory).
template <class T> struct IdxPtr {
  T *base;
  const int *idx;
  int off;
  long long stride;
#ifdef __CUDACC__
  __device__ __forceinline__ T *get() const {
    return idx ? base + (long long)(*idx + off) * stride : base;
  }
#endif
};
template <class T> inline IdxPtr<T> plain_ptr(T *p) { return IdxPtr<T>{p, nullptr, 0, 0}; }

// ---------------------------------------------------------------- 1D factors
// Banded evaluation matrices of one direction: row i (collocation point tau_i)
// has W = p+1 stored entries at interior columns start[i] .. start[i]+W-1;
// band[o][i*W + t] = d^o B_{start[i]+t+1} / dxi^o (tau_i), zero where the
// column is a dropped boundary function.
struct Factor1D {
  int n_elem = 0, p = 0, n = 0, W = 0;
  std::vector<double> knots, tau;
  std::vector<int> start;
  std::vector<double> band[3];
  std::vector<double> lam;      // n, ascending
  std::vector<double> U, Vt;    // n x n row-major
  // device copies
  DevBuf<int> d_start;
  DevBuf<double> d_band[3];
  DevBuf<double> d_tau;
  DevBuf<double> d_lam;
  DevBuf<double> d_Vt, d_U;     // FP64 FD operands (row-major, ld = n)
  DevBuf<float> d_Vt32, d_U32;  // TF32 FD operands (row-major, ld = kpad)
  DevBuf<float> d_Vt32lo, d_U32lo;  // TF32 roundings of their remainders (the TF32X3 form)
  DevBuf<__nv_bfloat16> d_Vt16, d_U16;
  int kpad = 0;                 // padded leading dimension for the TC operands
  double cond_U = 0.0;
  double setup_solver_s = 0.0;  // time in the eigen-factorisation's locked (cuSOLVER) parts
  // Folded form of the FD factors (eigenvectors even or odd under i -> n-1-i): the
  // eigen-index reordered [even | odd], Bf (n x n, forward, block diagonal in the
  // folded basis), Bi (ne x n, inverse, pairs a / n-1-a), eigenvalues in that order.
  bool folded = false;
  int ne = 0;
  DevBuf<double> d_Bf, d_Bi, d_lam_fold;
  DevBuf<double> d_BfT, d_BiT;  // their transposes (n x n, n x ne), for the FMA kernel
  // FD pencil (K + shift B', M): shift = w_l, the wind of the direction (Sec. 3.2)
  double shift = 0.0;

  // Weighted-quadrature Galerkin data (scheme 1, Sec. 2.3).  Quadrature points xq (nq);
  // the interior basis and its first derivative at them, banded: point q touches the
  // interior functions qstart[q] .. qstart[q] + W - 1 (qband[b][q W + t]); the four
  // univariate rules w^{(s,t)}, banded: test function i has weights on the points
  // wstart[i] .. wstart[i] + WW - 1 (wband[2 s + t][i WW + u]); and the univariate
  // Galerkin matrices M = int B_i B_j, K = int B_i' B_j' of the FD pencil, banded with
  // width GW = 2p + 1 from column gstart[i] (eq. univariateWQ).
  int scheme = 0;
  int nq = 0, WW = 0, GW = 0;
  std::vector<double> xq;
  std::vector<int> qstart, wstart, gstart;
  std::vector<double> qband[2], wband[4], gM, gK;
  DevBuf<int> d_qstart, d_wstart;
  DevBuf<double> d_qband[2], d_wband[4], d_xq;
};

struct FdScale;
template <class Tout>
void launch_gemm_fp64_fold(int dir, IdxPtr<const double> A, const double *Bt, IdxPtr<Tout> out,
                           int M, int n, int ne, const FdScale *scale, cudaStream_t s, int nrhs);
// The folded products on FP64 FMAs (kernels_fd64_fma.cu): BT is d_BfT (dir 0) or d_BiT
// (dir 1); dinv (forward only, may be null) is the fused diagonal.
void launch_gemm_fp64_fold_fma(int dir, IdxPtr<const double> A, const double *BT,
                               IdxPtr<double> out, int M, int n, int ne, const double *dinv,
                               cudaStream_t s, int nrhs);
// The precision forms whose FD runs on the tensor cores (TF32, BF16, error-compensated TF32).
inline bool tensor_core_prec(int prec) {
  return prec == IGA_PREC_TF32 || prec == IGA_PREC_BF16 || prec == IGA_PREC_TF32X3;
}
// Whether the folded FP64 products of M rows of length n run on the FMA kernel (else on
// mma.sync); IGA_FD64=fma|mma forces one.
bool use_fold_fma(long long M, int n);
template <class Tout>
void launch_gemm_fp64_dense_mma(IdxPtr<const double> A, const double *Bt, IdxPtr<Tout> out,
                                int M, int n, const FdScale *scale, cudaStream_t s, int nrhs);

// 1D factors of (n_elem, p) with the FD pencil (K + shift B', M), cached per device;
// scheme 1: the weighted-quadrature Galerkin data and the Galerkin pencil (K^wq, M^wq).
std::shared_ptr<Factor1D> get_factor(int n_elem, int p, cudaStream_t stream, double shift = 0.0,
                                     int scheme = 0);
void build_basis_1d(Factor1D &f);  // host part (knots, tau, bands)
void build_wq_1d(Factor1D &f);     // host part of the WQ data (needs the knots)
int find_span(const std::vector<double> &t, int p, int m, double x);
void span_basis(const std::vector<double> &t, int p, int mu, double x, double out[3][kMaxBand]);

// Operations that touch device-wide state share one process-wide reader-writer lock, so
// that setups on several host threads never disturb another thread's stream capture:
// captures of solve graphs and kernel attribute changes hold it exclusively; the cuSOLVER
// eigensolves (which may load library code on first use) and the tensor-core autotuner
// hold it shared, so those of different shapes run concurrently but never while a capture
// is in progress.  Every kernel of this library is loaded once per device before
// the first problem is set up, so none of it is loaded during a capture.
DeviceLock &device_mutex();
// IGA_VERBOSE=2 prints the duration of each setup phase to stderr (0 when unset)
int verbose_level();
double wall_seconds();
void ensure_kernels_loaded();
void preload_kernels_fd64();
void preload_kernels_fd64_fma();
void preload_kernels_fd_tc();
void preload_kernels_fd_f64tc();
void preload_kernels_geom_op();
void preload_kernels_krylov();
void preload_kernels_bicgstab();

// ---------------------------------------------------------------- geometry
// Coefficient fields of L u_hat = sum_f q_f(x) * (derivative f of u_hat):
// 2D: f = 11, 22, 12, 1, 2          3D: 11, 22, 33, 12, 13, 23, 1, 2, 3
// q_aa = -G^{aa}, q_ab = -2 G^{ab} (a<b), q_c = -L_c.
constexpr int kMaxFields = 9;
struct FieldDesc {
  int order[kMaxDim];  // derivative order per direction
};
int num_fields(int d);
FieldDesc field_desc(int d, int f);

// ---------------------------------------------------------------- launches
struct BandDev {
  const int *start;
  const double *band0, *band1, *band2;
  int n, W;
};

void launch_geometry_fields(int d, const iga_geometry &g, const double *tau1, const double *tau2,
                            const double *tau3, int n1, int n2, int n3, double *fields,
                            long long ldf, cudaStream_t s);

// Banded mode product along direction dir (0-based) of an n1 x n2 x n3 tensor:
// out[o] = B^{(order[o])}_dir applied along dir, for o < nout.
// nrhs tensors stacked back to back (slowest index).
template <class Tin>
void launch_band_pass(IdxPtr<const Tin> in, double *const *outs, const int *orders, int nout,
                      int dir, int n1, int n2, int n3, const BandDev &b, cudaStream_t s,
                      int nrhs = 1);

// Several banded mode products along one direction in one launch: output q is
// B^{(orders[q])}_dir applied to ins[in_of[q]] (nin <= 3 FP64 inputs, nout <= 6 outputs);
// each input's taps are loaded once per point for all of its outputs.
void launch_band_pass_multi(const double *const *ins, int nin, double *const *outs,
                            const int *in_of, const int *orders, int nout, int dir, int n1, int n2,
                            int n3, const BandDev &b, cudaStream_t s, int nrhs = 1);

// Final pass along direction 0 with contraction by the coefficient fields:
// out = sum_t coef_t(x) * B^{(order_t)}_0 in[input_t].
struct ContractTerm {
  int input;  // index into ins
  int order;  // derivative order along direction 0
  const double *coef;
};
template <class Tin>
void launch_contract_pass(IdxPtr<const Tin> const *ins, const ContractTerm *terms, int nterm,
                          double *out, int n1, int n2, int n3, const BandDev &b, cudaStream_t s,
                          int nrhs = 1);

// FP64 mode-product GEMM with layout rotation:
//   out[r + M*c] (+scale) = sum_k A[r*K + k] * Bt[c*K + k],  r < M, c < N(=K).
// If lam != nullptr the result is divided by lam0[r % n0] + lam1[(r / n0) % n1] + lamc[c]
// (the FD diagonal, eq. FD2D / FD3D).
// The FD diagonal solve fused into a GEMM epilogue: either multiply by the
// precomputed reciprocal diagonal dinv (indexed like one right-hand side's output,
// i.e. the original DOF order), or divide by lam_r0[rl % n0] (+ lam_r1[rl / n0]) +
// lam_c[col] when dinv is null.
struct FdScale {
  const double *lam_r0, *lam_r1, *lam_c;  // lam_r1 may be null (2D)
  int n0;
  const double *dinv = nullptr;
};
// dinv[i] = 1 / (lambda_{i1} + lambda_{i2} (+ lambda_{i3})) for i in DOF order, in FP64
// and (if dinv32 != nullptr) FP32.
void launch_fd_diag_inverse(const double *lam, int n, int d, double *dinv, float *dinv32,
                            cudaStream_t s);
// the same with the eigenvalues of each direction (lam3 unused for d = 2)
void launch_fd_diag_inverse3(const double *lam1, const double *lam2, const double *lam3, int n,
                             int d, double *dinv, float *dinv32, cudaStream_t s);
// nrhs right-hand sides stacked as the slowest index (M = nrhs * rows per rhs).
template <class Tout>
void launch_gemm_fp64(IdxPtr<const double> A, const double *Bt, IdxPtr<Tout> out, int M, int N,
                      int K, const FdScale *scale, cudaStream_t s, int nrhs = 1);

// ---------------------------------------------------------------- weighted quadrature
// One launch of banded rectangular products along one direction (kernels_wq.cu): term t
// reads in[t] (nullptr: the pass input vin), applies band rows start[c] .. + width - 1 of
// the output coordinate c (values band + c * width), optionally times the pointwise
// field coef (on the input grid), and adds into output out_of[t].
constexpr int kWqMaxTerms = 9, kWqMaxOut = 9, kWqMaxFan = 3;
template <class Tin> struct WqPassArgs {
  IdxPtr<const Tin> vin;
  const Tin *in[kWqMaxTerms];
  const int *start[kWqMaxTerms];
  const double *band[kWqMaxTerms];
  const double *coef[kWqMaxTerms];
  int width[kWqMaxTerms];
  int out_of[kWqMaxTerms];
  double *out[kWqMaxOut];
  int nterm, nout;
  // fan-out pass (fan = 1): term t's band sum s is written, times the pointwise field
  // fcoef[t][k] on the output grid, to fout[t][k] for k < nfan[t] (out / out_of unused)
  int fan;
  int nfan[kWqMaxTerms];
  const double *fcoef[kWqMaxTerms][kWqMaxFan];
  double *fout[kWqMaxTerms][kWqMaxFan];
};
template <class Tin>
void launch_wq_pass(const WqPassArgs<Tin> &a, int dir, const int *ext_in, const int *ext_out,
                    int R, cudaStream_t s);
// Q = det(J) J^{-1} J^{-T} (eq. Q, K = I) at the tensor grid of WQ quadrature points:
// 2D fields (11, 22, 12), 3D (11, 22, 33, 12, 13, 23), then |det J|; fields[f * ldf + i].
void launch_wq_fields(int d, const iga_geometry &g, const double *x1, const double *x2,
                      const double *x3, int n1, int n2, int n3, double *fields, long long ldf,
                      cudaStream_t s);
void preload_kernels_wq();

// ---------------------------------------------------------------- Krylov kernels
struct RhsState {
  int done;         // this right-hand side has stopped iterating
  int flag;         // 0 running, 1 converged, 2 max_iter, 3 breakdown, 4 non-finite
  int kconv;        // Arnoldi steps taken by this right-hand side
  int pad;
  double bnorm, beta;
  double relres_true;
  double pad2;
};

struct SolveState {
  int k;            // Arnoldi step shared by all right-hand sides
  int kv;           // the step whose basis vector the third CGS2 pass writes (k before
                    // the Givens kernel, which runs beside that pass, advances it)
  int active;       // right-hand sides still iterating
  int max_iter;
  int R;
  double tol;
};

// Vectors of all right-hand sides are stored back to back: vector j of rhs r at
// V + (j R + r) N (same for Z); per-rhs small arrays at a fixed stride.
struct KrylovWs {
  double *V;
  void *Z;
  int z_fp32;
  double *H;                     // rhs r: H + r*hstride, (max_iter+1) x max_iter col-major
  long long hstride;
  double *cs, *sn;               // r * (max_iter + 1)
  double *g, *y, *hist;          // r * (max_iter + 2)
  double *partials;              // r * pstride, pstride = nblk * (max_iter + 2)
  long long pstride;
  unsigned int *counter;         // R last-block counters
  double *scal;                  // 8 per rhs
  SolveState *st;
  RhsState *rs;                  // R
  int nblk, R, max_iter;
  long long N;
};

int reduce_blocks(long long N, int mode);

// ---------------------------------------------------------------- BiCGStab
struct BicgState {
  double rho, rho_prev, alpha, omega;  // scalar recurrences
  double bnorm, tol, relres_true, pad;
  int k;         // current iteration (1-based)
  int steps;     // half steps taken: 2k - 1 after the BiCG half, 2k after the GMRES half
  int done;      // the loop has ended
  int flag;      // 0 converged, 2 max_iter, 3 breakdown (rho, (rhat, v) or (t, t) zero), 4 NaN
  int half;      // converged after the BiCG half of iteration k
  int max_iter;
  int pad2[2];
};

struct BicgWs {
  double *r, *rhat, *p, *v, *s, *t, *phat, *shat, *x;  // N each
  double *hist;      // ||residual|| / ||b|| at half steps 0 .. 2 max_iter
  double *partials;  // 3 x nblk
  unsigned int *counter;
  BicgState *st;
  long long N;
  int nblk;
};

void launch_bicg_init(const BicgWs &ws, const double *b, const double *r0, const double *x0,
                      cudaGraphConditionalHandle cond, int has_cond, cudaStream_t s);
void launch_bicg_p(const BicgWs &ws, cudaStream_t s);
void launch_bicg_alpha(const BicgWs &ws, cudaStream_t s);
void launch_bicg_s(const BicgWs &ws, cudaStream_t s);
void launch_bicg_omega(const BicgWs &ws, cudaStream_t s);
void launch_bicg_xr(const BicgWs &ws, cudaGraphConditionalHandle cond, int has_cond,
                    cudaStream_t s);
void launch_bicg_residual(const BicgWs &ws, const double *b, const double *Ax, cudaStream_t s);
void launch_init_solve(const KrylovWs &ws, const double *b, const double *r0,
                       cudaGraphConditionalHandle cond, int has_cond, cudaStream_t s);
// CGS2 in two parts: passes 1 and 2 (coefficients, the subdiagonal entry), then pass 3
// (the next basis vector), which may run beside the Givens kernel of the same step.
void launch_cgs2_coeffs(const KrylovWs &ws, double *w, cudaStream_t s);
void launch_cgs2_vector(const KrylovWs &ws, const double *w, cudaStream_t s);
// Pass 2 alone, after the operator's last pass fused with pass 1 (launch_cgs_pass1_op).
void launch_cgs2_pass2(const KrylovWs &ws, double *w, cudaStream_t s);
template <class Tin> struct ContractArgsT;
// The operator's final contraction (collocation) fused with CGS2 pass 1: w = the contraction
// of the direction-0 band products with the geometry fields, and h1 = V^T w, on the
// reduction passes' row partition.  Bitwise the same w and h1 as contract_pass_kernel
// followed by cgs_pass1_kernel.
void launch_cgs_pass1_op(const KrylovWs &ws, const ContractArgsT<double> &a, const BandDev &b,
                         int n, double *w, cudaStream_t s);
// IGA_FUSE_P1=0 keeps the operator's contraction and pass 1 as separate launches
bool fuse_pass1();
void launch_givens(const KrylovWs &ws, cudaGraphConditionalHandle cond, int has_cond,
                   cudaStream_t s);
void launch_finish(const KrylovWs &ws, const double *x0, int use_x0, double *x, cudaStream_t s);
void launch_residual_norm(const KrylovWs &ws, const double *b, const double *Ax, double *r,
                          cudaStream_t s);
void launch_axpby(const double *x, const double *y, double a, double b, double *out, long long N,
                  cudaStream_t s);

}  // namespace iga
