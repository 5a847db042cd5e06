// Problem context behind an iga_handle: factors, geometry fields, operator plan,
// FD buffers, Krylov workspace and the captured solve graphs.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <map>
#include <utility>

#include "iga_internal.h"

namespace iga {

void launch_field_maxabs(const double *fields, long long ldf, long long N, int nf,
                         unsigned long long *out, cudaStream_t s);

// tcgen05 FD (TF32 / BF16) -- defined in kernels_fd_tc.cu
struct TcFd;
TcFd *make_tc_fd(int d, int n, int precision, const Factor1D &f, cudaStream_t s, int R_max,
                 const float *dinv32);
void tc_fd_apply(TcFd &fd, IdxPtr<const double> in, IdxPtr<float> out, int R, cudaStream_t s);
void tc_fd_apply_f64out(TcFd &fd, IdxPtr<const double> in, double *out, int R, cudaStream_t s);
void destroy_tc_fd(TcFd *fd);
int *tc_fd_error_word(TcFd &fd);
struct TcFdDeleter {
  void operator()(TcFd *p) const { destroy_tc_fd(p); }
};

// The driver's cuTensorMapEncodeTiled (kernels_fd_tc.cu), for the tensor maps of both
// tensor-core FD paths.
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder();

// FP64 FD on exact BF16 slice products (IGA_PREC_FP64_TC) -- kernels_fd_f64tc.cu
struct F64TcFd;
bool f64tc_supported(int n);
F64TcFd *make_f64tc_fd(int d, int n, const Factor1D &f, cudaStream_t s, int R_max,
                       const double *dinv);
void f64tc_fd_apply(F64TcFd &fd, IdxPtr<const double> in, IdxPtr<double> out, int R,
                    cudaStream_t s);
void destroy_f64tc_fd(F64TcFd *fd);
int *f64tc_error_word(F64TcFd &fd);
struct F64TcFdDeleter {
  void operator()(F64TcFd *p) const { destroy_f64tc_fd(p); }
};

struct OpPlan {
  int nA = 0;
  int ordA[3] = {0, 0, 0};
  int nB = 0;
  int B_in[6] = {0, 0, 0, 0, 0, 0};
  int B_ord[6] = {0, 0, 0, 0, 0, 0};
  int nterm = 0;
  ContractTerm terms[kMaxFields];
};

// One launch of the weighted-quadrature operator (kernels_wq.cu): banded products along
// direction dir, either expansion onto the quadrature grid by the basis values /
// derivatives (kind 0, band selector = derivative order) or contraction back to the test
// functions by a univariate rule (kind 1, selector = 2 s + t).  Inputs and outputs are
// scratch slots (-1: the chain's input / output vector).
struct WqPass {
  int dir = 0, kind = 0;
  int ext_in[3] = {1, 1, 1}, ext_out[3] = {1, 1, 1};
  int nterm = 0, nout = 0;
  int in_slot[kWqMaxTerms] = {};
  int sel[kWqMaxTerms] = {};
  int coef[kWqMaxTerms] = {};
  int out_of[kWqMaxTerms] = {};
  int out_slot[kWqMaxOut] = {};
  // fan-out pass: term t writes its band sum times field fcoef[t][k] to slot fslot[t][k]
  int fan = 0;
  int nfan[kWqMaxTerms] = {};
  int fcoef[kWqMaxTerms][kWqMaxFan] = {};
  int fslot[kWqMaxTerms][kWqMaxFan] = {};
};

struct SolveGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches_fixed = 0, launches_iter = 0;
};

struct Ctx {
  int d = 0, n_elem = 0, p = 0, n = 0;
  long long N = 0;
  int scheme = 0;  // 0: collocation (Sec. 2.2), 1: weighted-quadrature Galerkin (Sec. 2.3)
  // weighted quadrature: nq points per direction, Nq = nq^d; Q fields (+ |det J|) on that
  // grid; the operator and load-vector pass chains and their scratch slots (per rhs)
  int nq = 0;
  long long Nq = 0, ldq = 0;
  int wq_nf = 0;
  bool wq_active[7] = {};
  DevBuf<double> wq_fields, wq_scratch;
  std::vector<WqPass> wq_op, wq_load;
  std::vector<long long> wq_slot_size;
  iga_geometry geom{};
  int prec = IGA_PREC_FP64;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::shared_ptr<Factor1D> fac;       // bands (operator) and the Poisson FD factors
  std::shared_ptr<Factor1D> facd[3];   // FD factors of each direction (pencil K + w_l B', M)
  bool fold_ok = false;                // one folded factor set serves every direction
  BandDev band{};

  DevBuf<double> fields;
  long long ldf = 0;
  int active[kMaxFields] = {};
  int nactive = 0;
  double field_maxabs[kMaxFields] = {};
  OpPlan plan;
  DevBuf<double> dinv;   // reciprocal FD diagonal 1/(lambda_i + mu_j (+ nu_k)), DOF order
  DevBuf<float> dinv32;  // the same in FP32 (tensor-core FD)

  // buffers sized for R_max right-hand sides
  int R_max = 0;
  DevBuf<double> op_scratch;  // (nA + nB) x R_max x N
  DevBuf<double> fd_scratch;  // 2 x R_max x N
  std::unique_ptr<TcFd, TcFdDeleter> tc;
  std::unique_ptr<F64TcFd, F64TcFdDeleter> f64tc;
  DevBuf<double> b, x, x0, w, r;

  // Krylov workspace for (ws_max_iter, ws_R)
  int ws_max_iter = 0, ws_R = 0;
  // launch shape of the reduction passes (iga_grid_mode); fixes their row partition
  int grid_mode = IGA_GRID_LATENCY;
  DevBuf<double> V, Zd, H, cs, sn, g, y, hist, partials, scal;
  DevBuf<float> Zf;
  DevBuf<unsigned int> counter;
  DevBuf<SolveState> st;
  DevBuf<RhsState> rs;
  KrylovWs ws{};
  SolveState *h_st = nullptr;  // pinned
  RhsState *h_rs = nullptr;    // pinned, R
  double *h_hist = nullptr;    // pinned, R x (max_iter + 2)

  // captured solve graphs keyed by (R, use_x0)
  std::map<std::pair<int, int>, SolveGraph> graphs;

  // BiCGStab (one right-hand side): r, rhat, p, v, s, t, phat, shat, the scalar state,
  // the residual history and the graphs keyed by use_x0
  int bicg_max_iter = 0;
  DevBuf<double> bicg_vec, bicg_hist, bicg_partials;
  DevBuf<unsigned int> bicg_counter;
  DevBuf<BicgState> bicg_st;
  BicgState *h_bicg = nullptr;    // pinned
  double *h_bicg_hist = nullptr;  // pinned, 2 bicg_max_iter + 1
  BicgWs bws{};
  std::map<int, SolveGraph> bicg_graphs;

  // the solve in flight (enqueue ... collect)
  bool pending = false;
  int pend_R = 0, pend_max_iter = 0;
  double pend_tol = 0.0;
  cudaEvent_t done_ev = nullptr;
  // an Arnoldi step forks the Givens kernel onto side_stream beside the last CGS2 pass
  cudaStream_t side_stream = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;

  ~Ctx();
  void setup(int d_, int n_elem_, int p_, const iga_geometry &g_, int prec_, cudaStream_t s_,
             int scheme_ = 0);
  void setup_wq();
  void setup_collocation_fields();
  void build_wq_plan();
  template <class Tin>
  void run_wq(const std::vector<WqPass> &chain, IdxPtr<const Tin> in, double *out, int R,
              cudaStream_t s);
  void wq_load_vector(const double *g, double *f, cudaStream_t s);
  void quadrature_points(double *xyz) const;
  double operator_flops() const;
  void ensure_capacity(int R);
  template <class Tin>
  void apply_operator(IdxPtr<const Tin> in, double *out, int R, cudaStream_t s);
  template <class Tin>
  void operator_passes(IdxPtr<const Tin> in, int R, cudaStream_t s, IdxPtr<const double> (&ins)[6]);
  template <class Tin>
  void operator_and_pass1(IdxPtr<const Tin> in, int R, cudaStream_t s);
  void precond(IdxPtr<const double> in, double *out, int R, cudaStream_t s);  // FP64 result
  void ensure_ws(int max_iter, int R);
  void launch_iteration(cudaGraphConditionalHandle cond, int has_cond, cudaStream_t s);
  void launch_solve_prologue(int use_x0, cudaGraphConditionalHandle cond, int has_cond,
                             cudaStream_t s);
  void launch_solve_epilogue(int use_x0, cudaStream_t s);
  SolveGraph &graph_for(int R, int use_x0);
  void drop_graphs();
  // Switch the reduction grid; the workspace (its partials are sized by the grid) and
  // the captured graphs are rebuilt on the next solve.
  void set_grid_mode(int mode) {
    if (mode == grid_mode) return;
    grid_mode = mode;
    drop_graphs();
    ws_max_iter = 0;
    ws_R = 0;
    bicg_max_iter = 0;
  }
  void ensure_bicg(int max_iter);
  void bicg_iteration(cudaGraphConditionalHandle cond, int has_cond, cudaStream_t s);
  void bicg_prologue(int use_x0, cudaGraphConditionalHandle cond, int has_cond, cudaStream_t s);
  void bicg_epilogue(cudaStream_t s);
  SolveGraph &bicg_graph_for(int use_x0);
  // Synchronous BiCGStab solve; half_steps = 2k or 2k - 1 (the paper's k or k - 0.5).
  iga_status solve_bicgstab(const double *rhs_dev, double *x_dev, int use_x0, double tol,
                            int max_iter, int *half_steps, double *hist_out, double *relres);
  void enqueue(int R, const double *rhs_dev, double *x_dev, int use_x0, double tol,
               int max_iter);
  bool ready();
  iga_status collect(int *iters, double *hist_out, double *relres, int *status_out);
  void collocation_points(double *xyz) const;
};

}  // namespace iga
