// Host orchestration: setup of a problem, the matrix-free operator plan, the FD
// chain of mode products, and GMRES as one CUDA graph whose Arnoldi loop is a
// device-side `while` conditional node (the Givens kernel ends the loop).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "context.h"

namespace iga {

Ctx::~Ctx() {
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  if (h_st) cudaFreeHost(h_st);
  if (h_hist) cudaFreeHost(h_hist);
}

// ------------------------------------------------------------------ setup
void Ctx::setup(int d_, int n_elem_, int p_, const iga_geometry &g_, int prec_, cudaStream_t s_) {
  d = d_;
  n_elem = n_elem_;
  p = p_;
  geom = g_;
  prec = prec_;
  stream = s_;
  fac = get_factor(n_elem, p, stream);
  n = fac->n;
  N = 1;
  for (int l = 0; l < d; ++l) N *= n;
  band = BandDev{fac->d_start.ptr, fac->d_band[0].ptr, fac->d_band[1].ptr, fac->d_band[2].ptr, n,
                 fac->W};
  IGA_CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));

  // geometry coefficient fields at the collocation points
  const int nf = num_fields(d);
  ldf = (N + 31) / 32 * 32;
  fields.alloc((size_t)nf * ldf);
  const double *tau = fac->d_tau.ptr;
  launch_geometry_fields(d, geom, tau, tau, tau, n, n, d == 3 ? n : 1, fields.ptr, ldf, stream);
  DevBuf<unsigned long long> dmax;
  dmax.alloc(nf);
  launch_field_maxabs(fields.ptr, ldf, N, nf, dmax.ptr, stream);
  unsigned long long hmax[kMaxFields];
  IGA_CUDA_TRY(cudaMemcpyAsync(hmax, dmax.ptr, nf * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, stream));
  IGA_CUDA_TRY(cudaStreamSynchronize(stream));
  double scale = 0.0;
  for (int f = 0; f < nf; ++f) {
    double v;
    std::memcpy(&v, &hmax[f], sizeof(double));
    field_maxabs[f] = v;
    if (!std::isfinite(v)) throw Error{IGA_ERR_INVALID_ARG, "geometry map is singular"};
    int ord = 0;
    for (int l = 0; l < d; ++l) ord += field_desc(d, f).order[l];
    if (ord == 2) scale = std::max(scale, v);
  }
  // A field is dropped when it vanishes identically up to rounding of the
  // general formula (e.g. G^{12} and L_2 on the annulus).
  nactive = 0;
  for (int f = 0; f < nf; ++f)
    if (field_maxabs[f] > 1e-12 * scale) active[nactive++] = f;

  // operator plan: passes along the slow directions first, contraction along dir 0
  plan = OpPlan{};
  auto find_or_add = [](int *arr, int &cnt, int v) {
    for (int q = 0; q < cnt; ++q)
      if (arr[q] == v) return q;
    arr[cnt] = v;
    return cnt++;
  };
  for (int a = 0; a < nactive; ++a) {
    const FieldDesc fd = field_desc(d, active[a]);
    int input;
    if (d == 2) {
      input = find_or_add(plan.ordA, plan.nA, fd.order[1]);
    } else {
      const int ia = find_or_add(plan.ordA, plan.nA, fd.order[2]);
      int q = 0;
      for (; q < plan.nB; ++q)
        if (plan.B_in[q] == ia && plan.B_ord[q] == fd.order[1]) break;
      if (q == plan.nB) {
        plan.B_in[q] = ia;
        plan.B_ord[q] = fd.order[1];
        plan.nB++;
      }
      input = q;
    }
    plan.terms[plan.nterm++] = ContractTerm{input, fd.order[0], fields.ptr + active[a] * ldf};
  }
  op_scratch.alloc((size_t)(plan.nA + plan.nB) * N);
  fd_scratch.alloc(2 * (size_t)N);
  b.alloc(N);
  x.alloc(N);
  x0.alloc(N);
  w.alloc(N);
  r.alloc(N);
  if (prec == IGA_PREC_TF32 || prec == IGA_PREC_BF16)
    tc.reset(make_tc_fd(d, n, prec, *fac, stream));
  IGA_CUDA_TRY(cudaStreamSynchronize(stream));
}

// ------------------------------------------------------------------ operator
template <class Tin>
void Ctx::apply_operator(IdxPtr<const Tin> in, double *out, cudaStream_t s) {
  double *TA[3], *TB[6];
  for (int q = 0; q < plan.nA; ++q) TA[q] = op_scratch.ptr + (size_t)q * N;
  for (int q = 0; q < plan.nB; ++q) TB[q] = op_scratch.ptr + (size_t)(plan.nA + q) * N;
  const int n3 = d == 3 ? n : 1;
  // first pass along the slowest direction (d-1) reads the input
  launch_band_pass<Tin>(in, TA, plan.ordA, plan.nA, d - 1, n, n, n3, band, s);
  IdxPtr<const double> ins[6];
  if (d == 2) {
    for (int q = 0; q < plan.nA; ++q) ins[q] = plain_ptr<const double>(TA[q]);
  } else {
    for (int a = 0; a < plan.nA; ++a) {
      double *outs[3];
      int ords[3], cnt = 0;
      for (int q = 0; q < plan.nB; ++q)
        if (plan.B_in[q] == a) {
          outs[cnt] = TB[q];
          ords[cnt] = plan.B_ord[q];
          ++cnt;
        }
      if (cnt)
        launch_band_pass<double>(plain_ptr<const double>(TA[a]), outs, ords, cnt, 1, n, n, n3,
                                 band, s);
    }
    for (int q = 0; q < plan.nB; ++q) ins[q] = plain_ptr<const double>(TB[q]);
  }
  launch_contract_pass<double>(ins, plan.terms, plan.nterm, out, n, n, n3, band, s);
}

template void Ctx::apply_operator<double>(IdxPtr<const double>, double *, cudaStream_t);
template void Ctx::apply_operator<float>(IdxPtr<const float>, double *, cudaStream_t);

// ------------------------------------------------------------------ FD (FP64)
template <class Tout>
static void fd_chain_fp64(const Ctx &c, IdxPtr<const double> in, IdxPtr<Tout> out, cudaStream_t s) {
  const Factor1D &f = *c.fac;
  const int n = c.n;
  double *t0 = c.fd_scratch.ptr, *t1 = c.fd_scratch.ptr + c.N;
  const int M = (int)(c.N / n);
  auto P = [](double *p) { return plain_ptr<double>(p); };
  auto Pc = [](const double *p) { return plain_ptr<const double>(p); };
  if (c.d == 2) {
    FdScale sc{f.d_lam.ptr, nullptr, f.d_lam.ptr, n};
    launch_gemm_fp64<double>(in, f.d_Vt.ptr, P(t0), M, n, n, nullptr, s);
    launch_gemm_fp64<double>(Pc(t0), f.d_Vt.ptr, P(t1), M, n, n, &sc, s);
    launch_gemm_fp64<double>(Pc(t1), f.d_U.ptr, P(t0), M, n, n, nullptr, s);
    launch_gemm_fp64<Tout>(Pc(t0), f.d_U.ptr, out, M, n, n, nullptr, s);
  } else {
    FdScale sc{f.d_lam.ptr, f.d_lam.ptr, f.d_lam.ptr, n};
    launch_gemm_fp64<double>(in, f.d_Vt.ptr, P(t0), M, n, n, nullptr, s);
    launch_gemm_fp64<double>(Pc(t0), f.d_Vt.ptr, P(t1), M, n, n, nullptr, s);
    launch_gemm_fp64<double>(Pc(t1), f.d_Vt.ptr, P(t0), M, n, n, &sc, s);
    launch_gemm_fp64<double>(Pc(t0), f.d_U.ptr, P(t1), M, n, n, nullptr, s);
    launch_gemm_fp64<double>(Pc(t1), f.d_U.ptr, P(t0), M, n, n, nullptr, s);
    launch_gemm_fp64<Tout>(Pc(t0), f.d_U.ptr, out, M, n, n, nullptr, s);
  }
}

void Ctx::precond(IdxPtr<const double> in, double *out, cudaStream_t s) {
  if (prec == IGA_PREC_NONE) {
    throw Error{IGA_ERR_INVALID_ARG, "precond on an unpreconditioned handle"};
  } else if (prec == IGA_PREC_FP64) {
    fd_chain_fp64<double>(*this, in, plain_ptr<double>(out), s);
  } else {
    tc_fd_apply_f64out(*tc, in, out, s);
  }
}

// ------------------------------------------------------------------ Krylov workspace
void Ctx::ensure_ws(int max_iter) {
  if (max_iter <= ws_max_iter) return;
  const long long ld = (N + 31) / 32 * 32;
  const int nblk = reduce_blocks(N);
  V.alloc((size_t)(max_iter + 1) * ld);
  if (prec == IGA_PREC_FP64) Zd.alloc((size_t)max_iter * ld);
  if (prec == IGA_PREC_TF32 || prec == IGA_PREC_BF16) Zf.alloc((size_t)max_iter * ld);
  H.alloc((size_t)(max_iter + 1) * max_iter);
  cs.alloc(max_iter + 1);
  sn.alloc(max_iter + 1);
  g.alloc(max_iter + 2);
  y.alloc(max_iter + 2);
  hist.alloc(max_iter + 2);
  partials.alloc((size_t)nblk * (max_iter + 2));
  scal.alloc(8);
  counter.alloc(4);
  st.alloc(1);
  IGA_CUDA_TRY(cudaMemsetAsync(counter.ptr, 0, 4 * sizeof(unsigned int), stream));
  IGA_CUDA_TRY(cudaMemsetAsync(H.ptr, 0, (size_t)(max_iter + 1) * max_iter * 8, stream));
  IGA_CUDA_TRY(cudaMemsetAsync(hist.ptr, 0, (size_t)(max_iter + 2) * 8, stream));
  if (h_st) cudaFreeHost(h_st);
  if (h_hist) cudaFreeHost(h_hist);
  h_st = nullptr;
  h_hist = nullptr;
  IGA_CUDA_TRY(cudaMallocHost(&h_st, sizeof(SolveState)));
  IGA_CUDA_TRY(cudaMallocHost(&h_hist, (size_t)(max_iter + 2) * 8));
  ws = KrylovWs{};
  ws.V = V.ptr;
  ws.ldv = ld;
  if (prec == IGA_PREC_FP64) {
    ws.Z = Zd.ptr;
    ws.ldz = ld;
    ws.z_fp32 = 0;
  } else if (prec == IGA_PREC_NONE) {
    ws.Z = V.ptr;  // P = I: z_k = v_k
    ws.ldz = ld;
    ws.z_fp32 = 0;
  } else {
    ws.Z = Zf.ptr;
    ws.ldz = ld;
    ws.z_fp32 = 1;
  }
  ws.H = H.ptr;
  ws.cs = cs.ptr;
  ws.sn = sn.ptr;
  ws.g = g.ptr;
  ws.y = y.ptr;
  ws.hist = hist.ptr;
  ws.partials = partials.ptr;
  ws.counter = counter.ptr;
  ws.scal = scal.ptr;
  ws.st = st.ptr;
  ws.nblk = nblk;
  ws.N = N;
  ws.max_iter = max_iter;
  ws_max_iter = max_iter;
  // the graph refers to the old buffers
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  gexec = nullptr;
  graph = nullptr;
  g_max_iter = -1;
}

// ------------------------------------------------------------------ GMRES steps
void Ctx::launch_iteration(cudaGraphConditionalHandle cond, int has_cond, cudaStream_t s) {
  const int *kptr = &ws.st->k;
  IdxPtr<const double> vk{ws.V, kptr, 0, ws.ldv};
  if (prec == IGA_PREC_NONE) {
    apply_operator<double>(vk, w.ptr, s);
  } else if (prec == IGA_PREC_FP64) {
    IdxPtr<double> zk{(double *)ws.Z, kptr, 0, ws.ldz};
    fd_chain_fp64<double>(*this, vk, zk, s);
    apply_operator<double>(IdxPtr<const double>{(const double *)ws.Z, kptr, 0, ws.ldz}, w.ptr, s);
  } else {
    IdxPtr<float> zk{(float *)ws.Z, kptr, 0, ws.ldz};
    tc_fd_apply(*tc, vk, zk, s);
    apply_operator<float>(IdxPtr<const float>{(const float *)ws.Z, kptr, 0, ws.ldz}, w.ptr, s);
  }
  launch_cgs2(ws, w.ptr, s);
  launch_givens(ws, cond, has_cond, s);
}

void Ctx::launch_solve_prologue(int use_x0, cudaGraphConditionalHandle cond, int has_cond,
                                cudaStream_t s) {
  const double *r0 = b.ptr;
  if (use_x0) {
    apply_operator<double>(plain_ptr<const double>(x0.ptr), w.ptr, s);
    launch_axpby(b.ptr, w.ptr, 1.0, -1.0, r.ptr, N, s);
    r0 = r.ptr;
  }
  launch_dot(b.ptr, b.ptr, N, ws, ws.scal + 0, s);
  launch_dot(r0, r0, N, ws, ws.scal + 1, s);
  launch_init_solve(ws, r0, cond, has_cond, s);
}

void Ctx::launch_solve_epilogue(int use_x0, cudaStream_t s) {
  launch_finish(ws, x0.ptr, use_x0, x.ptr, s);
  apply_operator<double>(plain_ptr<const double>(x.ptr), w.ptr, s);
  launch_residual_norm(ws, b.ptr, w.ptr, r.ptr, s);
}

void Ctx::build_graph(int max_iter, int use_x0) {
  // max_iter and tol live in device state, so one graph serves every solve
  if (gexec && g_use_x0 == use_x0) return;
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  gexec = nullptr;
  graph = nullptr;
  cudaStream_t s = cap_stream;
  IGA_CUDA_TRY(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  IGA_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
  IGA_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
  cudaGraph_t body = nullptr;
  const long long c0 = g_launch_count;
  try {
    launch_solve_prologue(use_x0, cond, 1, s);
    cudaStreamCaptureStatus cst;
    cudaGraph_t capg;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    IGA_CUDA_TRY(cudaStreamGetCaptureInfo(s, &cst, nullptr, &capg, &deps, nullptr, &ndeps));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t cnode;
    IGA_CUDA_TRY(cudaGraphAddNode(&cnode, capg, deps, nullptr, ndeps, &np));
    body = np.conditional.phGraph_out[0];
    IGA_CUDA_TRY(cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1,
                                                     cudaStreamSetCaptureDependencies));
    launch_solve_epilogue(use_x0, s);
  } catch (...) {
    cudaGraph_t dummy;
    cudaStreamEndCapture(s, &dummy);
    throw;
  }
  IGA_CUDA_TRY(cudaStreamEndCapture(s, &graph));
  const long long c1 = g_launch_count;
  IGA_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
  try {
    launch_iteration(cond, 1, s);
  } catch (...) {
    cudaGraph_t dummy;
    cudaStreamEndCapture(s, &dummy);
    throw;
  }
  IGA_CUDA_TRY(cudaStreamEndCapture(s, &body));
  launches_fixed = (int)(c1 - c0);
  launches_iter = (int)(g_launch_count - c1);
  IGA_CUDA_TRY(cudaGraphInstantiate(&gexec, graph, 0));
  g_max_iter = max_iter;
  g_use_x0 = use_x0;
}

static bool eager_mode() {
  const char *e = std::getenv("IGA_EAGER");
  return e && e[0] == '1';
}

iga_status Ctx::solve(const double *rhs_dev, double *x_dev, int use_x0, double tol, int max_iter,
                      int *iters, double *hist_out, double *relres) {
  ensure_ws(max_iter);
  SolveState hs{};
  hs.tol = tol;
  hs.max_iter = max_iter;
  *h_st = hs;
  IGA_CUDA_TRY(cudaMemcpyAsync(ws.st, h_st, sizeof(SolveState), cudaMemcpyHostToDevice, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(b.ptr, rhs_dev, N * 8, cudaMemcpyDeviceToDevice, stream));
  if (use_x0)
    IGA_CUDA_TRY(cudaMemcpyAsync(x0.ptr, x_dev, N * 8, cudaMemcpyDeviceToDevice, stream));
  if (!eager_mode()) {
    build_graph(max_iter, use_x0);
    IGA_CUDA_TRY(cudaGraphLaunch(gexec, stream));
  } else {
    launch_solve_prologue(use_x0, 0, 0, stream);
    for (int it = 0; it <= max_iter; ++it) {
      IGA_CUDA_TRY(cudaMemcpyAsync(h_st, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, stream));
      IGA_CUDA_TRY(cudaStreamSynchronize(stream));
      if (h_st->done) break;
      launch_iteration(0, 0, stream);
    }
    launch_solve_epilogue(use_x0, stream);
  }
  IGA_CUDA_TRY(cudaMemcpyAsync(x_dev, x.ptr, N * 8, cudaMemcpyDeviceToDevice, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(h_st, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(h_hist, ws.hist, (size_t)(max_iter + 1) * 8,
                               cudaMemcpyDeviceToHost, stream));
  IGA_CUDA_TRY(cudaStreamSynchronize(stream));
  if (tc) {
    int err = 0;
    IGA_CUDA_TRY(cudaMemcpy(&err, tc_fd_error_word(*tc), sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      IGA_CUDA_TRY(cudaMemset(tc_fd_error_word(*tc), 0, sizeof(int)));
      throw Error{IGA_ERR_DEVICE_TIMEOUT,
                  "a tensor-core FD wait timed out (code " + std::to_string(err) + ")"};
    }
  }
  const SolveState &r_ = *h_st;
  if (iters) *iters = r_.k;
  if (hist_out) {
    for (int j = 0; j <= r_.k && j <= max_iter; ++j) hist_out[j] = h_hist[j];
    for (int j = r_.k + 1; j <= max_iter; ++j) hist_out[j] = 0.0;
  }
  if (relres) *relres = r_.relres_true;
  if (r_.flag == 4 || !std::isfinite(r_.relres_true)) return IGA_ERR_NAN;
  if (r_.flag == 2 && tol > 0.0) return IGA_ERR_NO_CONVERGENCE;
  return IGA_OK;
}

// ------------------------------------------------------------------ points (host)
void Ctx::collocation_points(double *xyz) const {
  const std::vector<double> &tau = fac->tau;
  const double r0 = geom.r_inner, r1 = geom.r_outer, w_ = 0.5 * M_PI;
  const long long n3 = d == 3 ? n : 1;
  for (long long i3 = 0; i3 < n3; ++i3)
    for (long long i2 = 0; i2 < n; ++i2)
      for (long long i1 = 0; i1 < n; ++i1) {
        const long long i = i1 + n * (i2 + n * i3);
        const double xi = tau[i1], eta = tau[i2], zeta = d == 3 ? tau[i3] : 0.0;
        double P[3] = {xi, eta, zeta};
        if (geom.kind != IGA_GEOM_IDENTITY) {
          const double r = r0 + (r1 - r0) * xi;
          const double X = r * std::cos(w_ * eta), Y = r * std::sin(w_ * eta);
          P[0] = X;
          P[1] = Y;
          if (geom.kind == IGA_GEOM_REVOLVED_ANNULUS) {
            const double phi = w_ * zeta, a = X + 1.0, bb = 1.0;
            P[0] = -1.0 + a * std::cos(phi) + bb * std::sin(phi);
            P[2] = -1.0 - a * std::sin(phi) + bb * std::cos(phi);
          }
        }
        for (int l = 0; l < d; ++l) xyz[i * d + l] = P[l];
      }
}

}  // namespace iga
