// extern "C" boundary (include/iga_fd.h).  Every entry point converts internal
// exceptions into an iga_status and records a message for iga_last_error().
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "context.h"

struct iga_ctx {
  iga::Ctx c;
};

namespace iga {
static thread_local std::string g_last_error;
thread_local long long g_launch_count = 0;
void set_error(const std::string &msg) { g_last_error = msg; }
}  // namespace iga

template <class F> static iga_status guarded(F &&f) {
  try {
    iga::g_last_error.clear();
    return f();
  } catch (const iga::Error &e) {
    iga::set_error(e.msg);
    return e.status;
  } catch (const std::bad_alloc &) {
    iga::set_error("host allocation failed");
    return IGA_ERR_OOM;
  } catch (const std::exception &e) {
    iga::set_error(e.what());
    return IGA_ERR_CUDA;
  }
}

extern "C" {

iga_status iga_setup(int d, int n_elem, int p, const iga_geometry *geom, int precision,
                     void *stream, iga_handle *out) {
  return iga_setup_scheme(d, n_elem, p, geom, IGA_SCHEME_COLLOCATION, precision, stream, out);
}

iga_status iga_setup_scheme(int d, int n_elem, int p, const iga_geometry *geom, int scheme,
                            int precision, void *stream, iga_handle *out) {
  return guarded([&]() -> iga_status {
    if (!out || !geom) throw iga::Error{IGA_ERR_INVALID_ARG, "null pointer argument"};
    *out = nullptr;
    if (d != 2 && d != 3) throw iga::Error{IGA_ERR_INVALID_ARG, "d must be 2 or 3"};
    if (p < 2 || p > iga::kMaxDeg) throw iga::Error{IGA_ERR_INVALID_ARG, "p must be in 2..6"};
    if (n_elem < 3 || n_elem > 4096)
      throw iga::Error{IGA_ERR_INVALID_ARG, "n_elem must be in 3..4096"};
    if (precision < IGA_PREC_FP64 || precision > IGA_PREC_FP64_TC)
      throw iga::Error{IGA_ERR_INVALID_ARG, "bad precision"};
    if (scheme != IGA_SCHEME_COLLOCATION && scheme != IGA_SCHEME_WQ_GALERKIN)
      throw iga::Error{IGA_ERR_INVALID_ARG, "bad discretization scheme"};
    if (geom->kind < IGA_GEOM_IDENTITY || geom->kind > IGA_GEOM_REVOLVED_ANNULUS)
      throw iga::Error{IGA_ERR_INVALID_ARG, "bad geometry kind"};
    if (geom->kind != IGA_GEOM_IDENTITY &&
        !(geom->r_inner > 0.0 && geom->r_outer > geom->r_inner && std::isfinite(geom->r_outer)))
      throw iga::Error{IGA_ERR_INVALID_ARG, "need 0 < r_inner < r_outer"};
    if (geom->kind == IGA_GEOM_REVOLVED_ANNULUS && d != 3)
      throw iga::Error{IGA_ERR_INVALID_ARG, "the revolved ring is 3D"};
    for (int l = 0; l < d; ++l)
      if (!std::isfinite(geom->wind[l])) throw iga::Error{IGA_ERR_INVALID_ARG, "wind must be finite"};
    const double n = n_elem + p - 2;
    if (std::pow(n, d) > 2.0e9) throw iga::Error{IGA_ERR_INVALID_ARG, "problem too large"};
    if (scheme == IGA_SCHEME_WQ_GALERKIN) {
      // the quadrature grid has about 2 n_elem points per direction
      const double nq = 2.0 * n_elem + 2.0 * p + 1.0;
      if (std::pow(nq, d) > 2.0e9) throw iga::Error{IGA_ERR_INVALID_ARG, "problem too large"};
    }
    iga_ctx *h = new iga_ctx();
    try {
      h->c.setup(d, n_elem, p, *geom, precision, (cudaStream_t)stream, scheme);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
    return IGA_OK;
  });
}

iga_status iga_dims(iga_handle h, int *n, long long *N) {
  return guarded([&]() -> iga_status {
    if (!h) throw iga::Error{IGA_ERR_INVALID_ARG, "null handle"};
    if (n) *n = h->c.n;
    if (N) *N = h->c.N;
    return IGA_OK;
  });
}

iga_status iga_collocation_points(iga_handle h, double *xyz_host) {
  return guarded([&]() -> iga_status {
    if (!h || !xyz_host) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    h->c.collocation_points(xyz_host);
    return IGA_OK;
  });
}

iga_status iga_quadrature_dims(iga_handle h, int *nq, long long *Nq) {
  return guarded([&]() -> iga_status {
    if (!h) throw iga::Error{IGA_ERR_INVALID_ARG, "null handle"};
    if (h->c.scheme != IGA_SCHEME_WQ_GALERKIN)
      throw iga::Error{IGA_ERR_UNSUPPORTED, "not a weighted-quadrature problem"};
    if (nq) *nq = h->c.nq;
    if (Nq) *Nq = h->c.Nq;
    return IGA_OK;
  });
}

iga_status iga_quadrature_points(iga_handle h, double *xyz_host) {
  return guarded([&]() -> iga_status {
    if (!h || !xyz_host) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    if (h->c.scheme != IGA_SCHEME_WQ_GALERKIN)
      throw iga::Error{IGA_ERR_UNSUPPORTED, "not a weighted-quadrature problem"};
    h->c.quadrature_points(xyz_host);
    return IGA_OK;
  });
}

iga_status iga_wq_load(iga_handle h, const double *g_dev, double *f_dev) {
  return guarded([&]() -> iga_status {
    if (!h || !g_dev || !f_dev) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    h->c.wq_load_vector(g_dev, f_dev, h->c.stream);
    return IGA_OK;
  });
}

iga_status iga_get_factor(iga_handle h, int dir, int which, double *out_host) {
  return guarded([&]() -> iga_status {
    if (!h || !out_host) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    if (dir < 0 || dir >= h->c.d) throw iga::Error{IGA_ERR_INVALID_ARG, "bad direction"};
    const iga::Factor1D &f = *h->c.fac;            // collocation factors
    const iga::Factor1D &fd = *h->c.facd[dir];     // FD factors of this direction
    const int n = f.n, W = f.W;
    auto dense = [&](int o, double sign) {
      std::memset(out_host, 0, sizeof(double) * n * n);
      for (int i = 0; i < n; ++i)
        for (int t = 0; t < W; ++t)
          out_host[(size_t)i * n + f.start[i] + t] = sign * f.band[o][(size_t)i * W + t];
    };
    auto gdense = [&](const std::vector<double> &band) {  // WQ Galerkin factor, banded
      std::memset(out_host, 0, sizeof(double) * n * n);
      for (int i = 0; i < n; ++i)
        for (int t = 0; t < f.GW; ++t)
          out_host[(size_t)i * n + f.gstart[i] + t] = band[(size_t)i * f.GW + t];
    };
    const bool wq = h->c.scheme == IGA_SCHEME_WQ_GALERKIN;
    switch (which) {
      case IGA_FACTOR_TAU: std::memcpy(out_host, f.tau.data(), sizeof(double) * n); break;
      case IGA_FACTOR_M:
        if (wq) gdense(f.gM); else dense(0, 1.0);
        break;
      case IGA_FACTOR_B1: dense(1, 1.0); break;
      case IGA_FACTOR_K:
        if (wq) gdense(f.gK); else dense(2, -1.0);
        break;
      case IGA_FACTOR_LAMBDA: std::memcpy(out_host, fd.lam.data(), sizeof(double) * n); break;
      case IGA_FACTOR_U: std::memcpy(out_host, fd.U.data(), sizeof(double) * n * n); break;
      case IGA_FACTOR_VT: std::memcpy(out_host, fd.Vt.data(), sizeof(double) * n * n); break;
      default: throw iga::Error{IGA_ERR_INVALID_ARG, "bad factor selector"};
    }
    return IGA_OK;
  });
}

iga_status iga_apply_operator(iga_handle h, const double *u_dev, double *Au_dev) {
  return guarded([&]() -> iga_status {
    if (!h || !u_dev || !Au_dev) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    h->c.apply_operator<double>(iga::plain_ptr<const double>(u_dev), Au_dev, 1, h->c.stream);
    return IGA_OK;
  });
}

iga_status iga_precond_apply(iga_handle h, const double *b_dev, double *s_dev) {
  return guarded([&]() -> iga_status {
    if (!h || !b_dev || !s_dev) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    if (h->c.prec == IGA_PREC_NONE) {
      IGA_CUDA_TRY(cudaMemcpyAsync(s_dev, b_dev, h->c.N * 8, cudaMemcpyDeviceToDevice,
                                   h->c.stream));
      return IGA_OK;
    }
    h->c.precond(iga::plain_ptr<const double>(b_dev), s_dev, 1, h->c.stream);
    return IGA_OK;
  });
}

static void check_solve_args(int nrhs, int max_iter, double tol) {
  if (nrhs < 1 || nrhs > 1024) throw iga::Error{IGA_ERR_INVALID_ARG, "nrhs must be in 1..1024"};
  if (max_iter < 1 || max_iter > iga::kMaxIter)
    throw iga::Error{IGA_ERR_INVALID_ARG, "max_iter must be in 1..4096"};
  if (!(tol >= 0.0)) throw iga::Error{IGA_ERR_INVALID_ARG, "tol must be >= 0"};
}

iga_status iga_solve(iga_handle h, const double *rhs_dev, double *x_dev, int use_x0, double tol,
                     int max_iter, int *iters, double *res_hist_host, double *true_relres) {
  return guarded([&]() -> iga_status {
    if (!h || !rhs_dev || !x_dev) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    check_solve_args(1, max_iter, tol);
    h->c.enqueue(1, rhs_dev, x_dev, use_x0 ? 1 : 0, tol, max_iter);
    return h->c.collect(iters, res_hist_host, true_relres, nullptr);
  });
}

iga_status iga_solve_multi(iga_handle h, int nrhs, const double *rhs_dev, double *x_dev,
                           int use_x0, double tol, int max_iter, int *iters,
                           double *res_hist_host, double *true_relres, int *status) {
  return guarded([&]() -> iga_status {
    if (!h || !rhs_dev || !x_dev) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    check_solve_args(nrhs, max_iter, tol);
    h->c.enqueue(nrhs, rhs_dev, x_dev, use_x0 ? 1 : 0, tol, max_iter);
    return h->c.collect(iters, res_hist_host, true_relres, status);
  });
}

iga_status iga_solve_async(iga_handle h, int nrhs, const double *rhs_dev, double *x_dev,
                           int use_x0, double tol, int max_iter) {
  return guarded([&]() -> iga_status {
    if (!h || !rhs_dev || !x_dev) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    check_solve_args(nrhs, max_iter, tol);
    h->c.enqueue(nrhs, rhs_dev, x_dev, use_x0 ? 1 : 0, tol, max_iter);
    return IGA_OK;
  });
}

iga_status iga_solve_ready(iga_handle h, int *ready) {
  return guarded([&]() -> iga_status {
    if (!h || !ready) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    *ready = h->c.ready() ? 1 : 0;
    return IGA_OK;
  });
}

iga_status iga_solve_collect(iga_handle h, int *iters, double *res_hist_host, double *true_relres,
                             int *status) {
  return guarded([&]() -> iga_status {
    if (!h) throw iga::Error{IGA_ERR_INVALID_ARG, "null handle"};
    return h->c.collect(iters, res_hist_host, true_relres, status);
  });
}

iga_status iga_solve_batched(int nprob, const iga_handle *handles, const int *nrhs,
                             const double *const *rhs_dev, double *const *x_dev, double tol,
                             int max_iter, int *iters, double *res_hist_host, double *true_relres,
                             int *status) {
  return guarded([&]() -> iga_status {
    if (nprob < 1 || !handles || !nrhs || !rhs_dev || !x_dev)
      throw iga::Error{IGA_ERR_INVALID_ARG, "bad batch arguments"};
    for (int q = 0; q < nprob; ++q) {
      if (!handles[q] || !rhs_dev[q] || !x_dev[q])
        throw iga::Error{IGA_ERR_INVALID_ARG, "null entry in batch"};
      check_solve_args(nrhs[q], max_iter, tol);
      for (int q2 = 0; q2 < q; ++q2)
        if (handles[q2] == handles[q])
          throw iga::Error{IGA_ERR_INVALID_ARG, "a handle appears twice in one batch"};
    }
    // enqueue every problem on its own stream, then collect in order
    int enq = 0;
    iga_status overall = IGA_OK;
    try {
      for (; enq < nprob; ++enq)
        handles[enq]->c.enqueue(nrhs[enq], rhs_dev[enq], x_dev[enq], 0, tol, max_iter);
    } catch (...) {
      for (int q = 0; q < enq; ++q) {
        try {
          handles[q]->c.collect(nullptr, nullptr, nullptr, nullptr);
        } catch (...) {
        }
      }
      throw;
    }
    long long off = 0;
    for (int q = 0; q < nprob; ++q) {
      const iga_status st = handles[q]->c.collect(
          iters ? iters + off : nullptr,
          res_hist_host ? res_hist_host + (size_t)off * (max_iter + 1) : nullptr,
          true_relres ? true_relres + off : nullptr, status ? status + off : nullptr);
      if (st == IGA_ERR_NAN) overall = IGA_ERR_NAN;
      else if (st != IGA_OK && overall == IGA_OK) overall = st;
      off += nrhs[q];
    }
    return overall;
  });
}

iga_status iga_solve_host(iga_handle h, const double *rhs_host, double *x_host, double tol,
                          int max_iter, int *iters, double *res_hist_host, double *true_relres) {
  return guarded([&]() -> iga_status {
    if (!h || !rhs_host || !x_host) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    check_solve_args(1, max_iter, tol);
    iga::Ctx &c = h->c;
    c.ensure_ws(max_iter, 1);
    IGA_CUDA_TRY(cudaMemcpyAsync(c.r.ptr, rhs_host, c.N * 8, cudaMemcpyHostToDevice, c.stream));
    // the solve copies rhs from c.r into c.b before it uses c.r as scratch
    c.enqueue(1, c.r.ptr, c.x0.ptr, 0, tol, max_iter);
    IGA_CUDA_TRY(cudaMemcpyAsync(x_host, c.x.ptr, c.N * 8, cudaMemcpyDeviceToHost, c.stream));
    return c.collect(iters, res_hist_host, true_relres, nullptr);
  });
}

iga_status iga_launch_counts(iga_handle h, int *fixed, int *per_iteration) {
  return guarded([&]() -> iga_status {
    if (!h) throw iga::Error{IGA_ERR_INVALID_ARG, "null handle"};
    iga::Ctx &c = h->c;
    c.ensure_ws(std::max(c.ws_max_iter, 1), 1);
    iga::SolveGraph &g = c.graph_for(1, 0);
    if (fixed) *fixed = g.launches_fixed;
    if (per_iteration) *per_iteration = g.launches_iter;
    return IGA_OK;
  });
}

iga_status iga_fd_kernel(iga_handle h, int nrhs, int *kind) {
  return guarded([&]() -> iga_status {
    if (!h || !kind || nrhs < 1) throw iga::Error{IGA_ERR_INVALID_ARG, "null handle or kind, or nrhs < 1"};
    const iga::Ctx &c = h->c;
    if (c.prec == IGA_PREC_NONE)
      throw iga::Error{IGA_ERR_INVALID_ARG, "unpreconditioned handle"};
    if (c.prec == IGA_PREC_FP64_TC) *kind = IGA_FD_KERNEL_FP64_SLICES;
    else if (c.prec != IGA_PREC_FP64) *kind = IGA_FD_KERNEL_TENSOR_CORE;
    else if (!c.fold_ok) *kind = IGA_FD_KERNEL_DENSE_MMA;
    else
      *kind = iga::use_fold_fma((long long)nrhs * (c.N / c.n), c.n) ? IGA_FD_KERNEL_FOLD_FMA
                                                                   : IGA_FD_KERNEL_FOLD_MMA;
    return IGA_OK;
  });
}

iga_status iga_operator_flops(iga_handle h, double *flops) {
  return guarded([&]() -> iga_status {
    if (!h || !flops) throw iga::Error{IGA_ERR_INVALID_ARG, "null handle or flops"};
    *flops = h->c.operator_flops();
    return IGA_OK;
  });
}

iga_status iga_solve_bicgstab(iga_handle h, const double *rhs_dev, double *x_dev, int use_x0,
                              double tol, int max_iter, int *half_steps, double *res_hist_host,
                              double *true_relres) {
  return guarded([&]() -> iga_status {
    if (!h || !rhs_dev || !x_dev) throw iga::Error{IGA_ERR_INVALID_ARG, "null argument"};
    check_solve_args(1, max_iter, tol);
    return h->c.solve_bicgstab(rhs_dev, x_dev, use_x0 ? 1 : 0, tol, max_iter, half_steps,
                               res_hist_host, true_relres);
  });
}

iga_status iga_set_grid_mode(iga_handle h, iga_grid_mode mode) {
  return guarded([&]() -> iga_status {
    if (!h) throw iga::Error{IGA_ERR_INVALID_ARG, "null handle"};
    if (mode != IGA_GRID_LATENCY && mode != IGA_GRID_THROUGHPUT)
      throw iga::Error{IGA_ERR_INVALID_ARG, "unknown grid mode"};
    iga::Ctx &c = h->c;
    if (c.pending) throw iga::Error{IGA_ERR_INVALID_ARG, "a solve is in flight on this handle"};
    c.set_grid_mode((int)mode);
    return IGA_OK;
  });
}

iga_status iga_prepare(iga_handle h, int nrhs, int max_iter) {
  return guarded([&]() -> iga_status {
    if (!h) throw iga::Error{IGA_ERR_INVALID_ARG, "null handle"};
    check_solve_args(nrhs, max_iter, 0.0);
    iga::Ctx &c = h->c;
    if (c.pending) throw iga::Error{IGA_ERR_INVALID_ARG, "a solve is in flight on this handle"};
    c.ensure_ws(max_iter, nrhs);
    c.graph_for(nrhs, 0);
    IGA_CUDA_TRY(cudaStreamSynchronize(c.stream));
    return IGA_OK;
  });
}

iga_status iga_test_set_device_error(iga_handle h, int code) {
  return guarded([&]() -> iga_status {
    if (!h) throw iga::Error{IGA_ERR_INVALID_ARG, "null handle"};
    iga::Ctx &c = h->c;
    int *ew = c.tc ? iga::tc_fd_error_word(*c.tc)
                   : c.f64tc ? iga::f64tc_error_word(*c.f64tc) : nullptr;
    if (!ew) throw iga::Error{IGA_ERR_INVALID_ARG, "the handle has no tensor-core FD"};
    if (c.pending) throw iga::Error{IGA_ERR_INVALID_ARG, "a solve is in flight on this handle"};
    IGA_CUDA_TRY(cudaMemcpyAsync(ew, &code, sizeof(int), cudaMemcpyHostToDevice, c.stream));
    IGA_CUDA_TRY(cudaStreamSynchronize(c.stream));
    return IGA_OK;
  });
}

iga_status iga_destroy(iga_handle h) {
  return guarded([&]() -> iga_status {
    delete h;
    return IGA_OK;
  });
}

const char *iga_status_string(iga_status s) {
  switch (s) {
    case IGA_OK: return "ok";
    case IGA_ERR_INVALID_ARG: return "invalid argument";
    case IGA_ERR_OOM: return "out of memory";
    case IGA_ERR_CUDA: return "CUDA error";
    case IGA_ERR_NOT_DIAGONALIZABLE: return "pencil not diagonalizable with real spectrum";
    case IGA_ERR_NO_CONVERGENCE: return "no convergence within max_iter";
    case IGA_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case IGA_ERR_NAN: return "non-finite value";
    case IGA_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *iga_last_error(void) { return iga::g_last_error.c_str(); }

}  // extern "C"
