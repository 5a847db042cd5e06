// BiCGStab with the FD preconditioner (Sec. 5's solver), one right-hand side, as one
// CUDA graph: prologue (r0, norms), a device-side `while` conditional node whose body
// is one BiCGStab iteration (two FD solves, two operator applications and the vector
// and scalar updates of kernels_bicgstab.cu; bicg_xr ends the loop), and the epilogue
// (FP64 true residual).  IGA_EAGER=1 runs the same kernels from a host loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "context.h"

namespace iga {

void Ctx::ensure_bicg(int max_iter) {
  ensure_capacity(1);
  if (max_iter <= bicg_max_iter) return;
  for (auto &kv : bicg_graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  bicg_graphs.clear();
  const int nblk = reduce_blocks(N, grid_mode);
  bicg_vec.alloc((size_t)8 * N);
  bicg_hist.alloc((size_t)2 * max_iter + 2);
  bicg_partials.alloc((size_t)3 * nblk);
  bicg_counter.alloc(1);
  bicg_st.alloc(1);
  IGA_CUDA_TRY(cudaMemsetAsync(bicg_counter.ptr, 0, sizeof(unsigned int), stream));
  if (h_bicg_hist) cudaFreeHost(h_bicg_hist);
  h_bicg_hist = nullptr;
  IGA_CUDA_TRY(cudaMallocHost(&h_bicg_hist, ((size_t)2 * max_iter + 2) * sizeof(double)));
  if (!h_bicg) IGA_CUDA_TRY(cudaMallocHost(&h_bicg, sizeof(BicgState)));
  double *v = bicg_vec.ptr;
  bws.r = v;
  bws.rhat = v + N;
  bws.p = v + 2 * N;
  bws.v = v + 3 * N;
  bws.s = v + 4 * N;
  bws.t = v + 5 * N;
  bws.phat = v + 6 * N;
  bws.shat = v + 7 * N;
  bws.x = x.ptr;
  bws.hist = bicg_hist.ptr;
  bws.partials = bicg_partials.ptr;
  bws.counter = bicg_counter.ptr;
  bws.st = bicg_st.ptr;
  bws.N = N;
  bws.nblk = nblk;
  bicg_max_iter = max_iter;
}

// z = M^{-1} y (FD in the handle's precision, FP64 result; identity when unpreconditioned)
static void bicg_precond(Ctx &c, const double *y, double *z, cudaStream_t s) {
  if (c.prec == IGA_PREC_NONE)
    IGA_CUDA_TRY(cudaMemcpyAsync(z, y, c.N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else
    c.precond(plain_ptr<const double>(y), z, 1, s);
}

void Ctx::bicg_iteration(cudaGraphConditionalHandle cond, int has_cond, cudaStream_t s) {
  launch_bicg_p(bws, s);
  bicg_precond(*this, bws.p, bws.phat, s);
  apply_operator<double>(plain_ptr<const double>(bws.phat), bws.v, 1, s);
  launch_bicg_alpha(bws, s);
  launch_bicg_s(bws, s);
  bicg_precond(*this, bws.s, bws.shat, s);
  apply_operator<double>(plain_ptr<const double>(bws.shat), bws.t, 1, s);
  launch_bicg_omega(bws, s);
  launch_bicg_xr(bws, cond, has_cond, s);
}

void Ctx::bicg_prologue(int use_x0, cudaGraphConditionalHandle cond, int has_cond,
                        cudaStream_t s) {
  const double *r0 = b.ptr;
  if (use_x0) {
    apply_operator<double>(plain_ptr<const double>(x0.ptr), w.ptr, 1, s);
    launch_axpby(b.ptr, w.ptr, 1.0, -1.0, r.ptr, N, s);
    r0 = r.ptr;
  }
  launch_bicg_init(bws, b.ptr, r0, use_x0 ? x0.ptr : nullptr, cond, has_cond, s);
}

void Ctx::bicg_epilogue(cudaStream_t s) {
  apply_operator<double>(plain_ptr<const double>(x.ptr), w.ptr, 1, s);
  launch_bicg_residual(bws, b.ptr, w.ptr, s);
}

SolveGraph &Ctx::bicg_graph_for(int use_x0) {
  auto it = bicg_graphs.find(use_x0);
  if (it != bicg_graphs.end()) return it->second;
  std::unique_lock<DeviceLock> dlk(device_mutex());
  SolveGraph sg;
  cudaStream_t s = cap_stream;
  IGA_CUDA_TRY(cudaGraphCreate(&sg.graph, 0));
  cudaGraphConditionalHandle cond;
  IGA_CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, sg.graph, 1, cudaGraphCondAssignDefault));
  IGA_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, sg.graph, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
  cudaGraph_t body = nullptr;
  const long long c0 = g_launch_count;
  try {
    bicg_prologue(use_x0, cond, 1, s);
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
    bicg_epilogue(s);
  } catch (...) {
    cudaGraph_t dummy;
    cudaStreamEndCapture(s, &dummy);
    cudaGraphDestroy(sg.graph);
    throw;
  }
  IGA_CUDA_TRY(cudaStreamEndCapture(s, &sg.graph));
  const long long c1 = g_launch_count;
  IGA_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
  try {
    bicg_iteration(cond, 1, s);
  } catch (...) {
    cudaGraph_t dummy;
    cudaStreamEndCapture(s, &dummy);
    cudaGraphDestroy(sg.graph);
    throw;
  }
  IGA_CUDA_TRY(cudaStreamEndCapture(s, &body));
  sg.launches_fixed = (int)(c1 - c0);
  sg.launches_iter = (int)(g_launch_count - c1);
  IGA_CUDA_TRY(cudaGraphInstantiate(&sg.exec, sg.graph, 0));
  return bicg_graphs[use_x0] = sg;
}

static bool bicg_eager() {
  const char *e = std::getenv("IGA_EAGER");
  return e && e[0] == '1';
}

iga_status Ctx::solve_bicgstab(const double *rhs_dev, double *x_dev, int use_x0, double tol,
                               int max_iter, int *half_steps, double *hist_out,
                               double *relres) {
  if (pending) throw Error{IGA_ERR_INVALID_ARG, "a solve is in flight on this handle"};
  ensure_bicg(max_iter);
  BicgState hs{};
  hs.tol = tol;
  hs.max_iter = max_iter;
  *h_bicg = hs;
  const size_t bytes = (size_t)N * 8;
  IGA_CUDA_TRY(cudaMemcpyAsync(bws.st, h_bicg, sizeof(BicgState), cudaMemcpyHostToDevice, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(b.ptr, rhs_dev, bytes, cudaMemcpyDeviceToDevice, stream));
  if (use_x0)
    IGA_CUDA_TRY(cudaMemcpyAsync(x0.ptr, x_dev, bytes, cudaMemcpyDeviceToDevice, stream));
  if (!bicg_eager()) {
    SolveGraph &sg = bicg_graph_for(use_x0);
    IGA_CUDA_TRY(cudaGraphLaunch(sg.exec, stream));
  } else {
    bicg_prologue(use_x0, 0, 0, stream);
    for (int it = 0; it < max_iter; ++it) {
      IGA_CUDA_TRY(cudaMemcpyAsync(h_bicg, bws.st, sizeof(BicgState), cudaMemcpyDeviceToHost,
                                   stream));
      IGA_CUDA_TRY(cudaStreamSynchronize(stream));
      if (h_bicg->done) break;
      bicg_iteration(0, 0, stream);
    }
    bicg_epilogue(stream);
  }
  IGA_CUDA_TRY(cudaMemcpyAsync(x_dev, x.ptr, bytes, cudaMemcpyDeviceToDevice, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(h_bicg, bws.st, sizeof(BicgState), cudaMemcpyDeviceToHost, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(h_bicg_hist, bws.hist, ((size_t)2 * max_iter + 1) * 8,
                               cudaMemcpyDeviceToHost, stream));
  IGA_CUDA_TRY(cudaStreamSynchronize(stream));
  const BicgState &st = *h_bicg;
  if (half_steps) *half_steps = st.steps;
  if (hist_out)
    for (int j = 0; j <= 2 * max_iter; ++j) hist_out[j] = j <= st.steps ? h_bicg_hist[j] : 0.0;
  if (relres) *relres = st.relres_true;
  if (st.flag == 4 || !std::isfinite(st.relres_true)) return IGA_ERR_NAN;
  if (st.flag == 3) {
    set_error("BiCGStab breakdown: rho, (rhat, v) or (t, t) became zero");
    return IGA_ERR_NO_CONVERGENCE;
  }
  if (st.flag == 2 && tol > 0.0) return IGA_ERR_NO_CONVERGENCE;
  return IGA_OK;
}

}  // namespace iga
