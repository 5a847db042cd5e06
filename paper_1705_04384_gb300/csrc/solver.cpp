// Host orchestration: setup of a problem, the matrix-free operator plan, the FD
// chain of mode products, and GMRES as one CUDA graph whose Arnoldi loop is a
// device-side `while` conditional node (the Givens kernel ends the loop).  R right-
// hand sides of one problem iterate in lockstep in the same graph: their vectors are
// stacked as the slowest index, so every operator pass and FD mode product serves all
// of them in one launch (coefficients and factors are read once for all R).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "context.h"
#include "contract_point.cuh"

#include <type_traits>

namespace iga {

Ctx::~Ctx() {
  if (pending && done_ev) cudaEventSynchronize(done_ev);
  drop_graphs();
  if (done_ev) cudaEventDestroy(done_ev);
  if (fork_ev) cudaEventDestroy(fork_ev);
  if (join_ev) cudaEventDestroy(join_ev);
  if (side_stream) cudaStreamDestroy(side_stream);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  if (h_st) cudaFreeHost(h_st);
  if (h_rs) cudaFreeHost(h_rs);
  if (h_hist) cudaFreeHost(h_hist);
  if (h_bicg) cudaFreeHost(h_bicg);
  if (h_bicg_hist) cudaFreeHost(h_bicg_hist);
}

void Ctx::drop_graphs() {
  for (auto &kv : graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  graphs.clear();
  for (auto &kv : bicg_graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  bicg_graphs.clear();
}

// ------------------------------------------------------------------ setup
void Ctx::setup(int d_, int n_elem_, int p_, const iga_geometry &g_, int prec_, cudaStream_t s_,
                int scheme_) {
  d = d_;
  n_elem = n_elem_;
  p = p_;
  geom = g_;
  prec = prec_;
  stream = s_;
  scheme = scheme_;
  const double t0 = wall_seconds();
  ensure_kernels_loaded();
  bool has_wind = false;
  for (int l = 0; l < d; ++l) has_wind = has_wind || geom.wind[l] != 0.0;
  if (has_wind && scheme == 1)
    throw Error{IGA_ERR_INVALID_ARG, "the weighted-quadrature scheme takes no wind"};
  fac = get_factor(n_elem, p, stream, 0.0, scheme);
  if (has_wind && (tensor_core_prec(prec) || prec == IGA_PREC_FP64_TC))
    throw Error{IGA_ERR_INVALID_ARG, "a wind requires precision FP64 or NONE"};
  if (prec == IGA_PREC_FP64_TC && !f64tc_supported(fac->n))
    throw Error{IGA_ERR_UNSUPPORTED, "precision FP64_TC takes n <= 148 basis functions per "
                                     "direction"};
  // per-direction FD factors: the pencil (K + w_l B', M) of Sec. 3.2 (w_l = 0: Poisson)
  for (int l = 0; l < 3; ++l)
    facd[l] = (l >= d || geom.wind[l] == 0.0) ? fac : get_factor(n_elem, p, stream, geom.wind[l]);
  fold_ok = fac->folded && !has_wind;
  n = fac->n;
  N = 1;
  for (int l = 0; l < d; ++l) N *= n;
  band = BandDev{fac->d_start.ptr, fac->d_band[0].ptr, fac->d_band[1].ptr, fac->d_band[2].ptr, n,
                 fac->W};
  IGA_CUDA_TRY(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
  IGA_CUDA_TRY(cudaEventCreateWithFlags(&done_ev, cudaEventDisableTiming));
  IGA_CUDA_TRY(cudaStreamCreateWithFlags(&side_stream, cudaStreamNonBlocking));
  IGA_CUDA_TRY(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
  IGA_CUDA_TRY(cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming));

  const double t1 = wall_seconds();
  if (scheme == 1) {
    setup_wq();
  } else {
    setup_collocation_fields();
  }
  const double t2 = wall_seconds();
  if (prec == IGA_PREC_FP64) {
    // the FP64 chain uses the folded eigen-order when one factor set with parity serves
    // every direction, else each direction's own eigenvalues
    dinv.alloc(N);
    if (fold_ok)
      launch_fd_diag_inverse(fac->d_lam_fold.ptr, n, d, dinv.ptr, nullptr, stream);
    else
      launch_fd_diag_inverse3(facd[0]->d_lam.ptr, facd[1]->d_lam.ptr, facd[2]->d_lam.ptr, n, d,
                              dinv.ptr, nullptr, stream);
  } else if (tensor_core_prec(prec)) {
    dinv32.alloc(N);
    launch_fd_diag_inverse(fac->d_lam.ptr, n, d, nullptr, dinv32.ptr, stream);
  } else if (prec == IGA_PREC_FP64_TC) {
    // the slice products use the unfolded factors (V^T, U) and eigen-order
    dinv.alloc(N);
    launch_fd_diag_inverse(fac->d_lam.ptr, n, d, dinv.ptr, nullptr, stream);
  }
  const double t3 = wall_seconds();
  ensure_capacity(1);
  IGA_CUDA_TRY(cudaStreamSynchronize(stream));
  if (verbose_level() >= 2)
    std::fprintf(stderr, "iga setup d=%d n=%d p=%d prec=%d: factors %.1f ms, fields %.1f ms, "
                 "diagonal %.1f ms, buffers and tensor-core context %.1f ms\n", d, n, p, prec,
                 1e3 * (t1 - t0), 1e3 * (t2 - t1), 1e3 * (t3 - t2), 1e3 * (wall_seconds() - t3));
}

// Geometry coefficient fields of the collocation operator and its pass plan.
void Ctx::setup_collocation_fields() {
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
}

// Buffers whose size scales with the number of right-hand sides.
void Ctx::ensure_capacity(int R) {
  if (R <= R_max) return;
  if (pending) throw Error{IGA_ERR_INVALID_ARG, "a solve is in flight on this handle"};
  drop_graphs();
  ws_max_iter = 0;  // the Krylov workspaces are rebuilt for the new capacity
  ws_R = 0;
  bicg_max_iter = 0;
  if (scheme == 1) {
    long long per = 0;
    for (long long sz : wq_slot_size) per += sz;
    wq_scratch.alloc((size_t)per * R);
  } else {
    op_scratch.alloc((size_t)(plan.nA + plan.nB) * R * N);
  }
  fd_scratch.alloc(2 * (size_t)R * N);
  b.alloc((size_t)R * N);
  x.alloc((size_t)R * N);
  x0.alloc((size_t)R * N);
  w.alloc((size_t)R * N);
  r.alloc((size_t)R * N);
  if (tensor_core_prec(prec)) {
    tc.reset();
    R_max = 0;  // until the new tensor-core context exists
    tc.reset(make_tc_fd(d, n, prec, *fac, stream, R, dinv32.ptr));
  }
  if (prec == IGA_PREC_FP64_TC) {
    f64tc.reset();
    R_max = 0;
    f64tc.reset(make_f64tc_fd(d, n, *fac, stream, R, dinv.ptr));
  }
  R_max = R;
}

// ------------------------------------------------------------------ operator
template <class Tin>
void Ctx::apply_operator(IdxPtr<const Tin> in, double *out, int R, cudaStream_t s) {
  if (scheme == 1) {  // weighted-quadrature Galerkin, eq. (WQapprox)
    run_wq<Tin>(wq_op, in, out, R, s);
    return;
  }
  IdxPtr<const double> ins[6];
  operator_passes<Tin>(in, R, s, ins);
  launch_contract_pass<double>(ins, plan.terms, plan.nterm, out, n, n, d == 3 ? n : 1, band, s, R);
}

// The band passes of the collocation operator before its final contraction (which reads
// ins): along direction d-1, then (3D) all second-direction passes in one launch.
template <class Tin>
void Ctx::operator_passes(IdxPtr<const Tin> in, int R, cudaStream_t s,
                          IdxPtr<const double> (&ins)[6]) {
  double *TA[3], *TB[6];
  const size_t blk = (size_t)R * N;
  for (int q = 0; q < plan.nA; ++q) TA[q] = op_scratch.ptr + q * blk;
  for (int q = 0; q < plan.nB; ++q) TB[q] = op_scratch.ptr + (plan.nA + q) * blk;
  const int n3 = d == 3 ? n : 1;
  // first pass along the slowest direction (d-1) reads the input
  launch_band_pass<Tin>(in, TA, plan.ordA, plan.nA, d - 1, n, n, n3, band, s, R);
  if (d == 2) {
    for (int q = 0; q < plan.nA; ++q) ins[q] = plain_ptr<const double>(TA[q]);
  } else {
    // all second-direction passes in one launch
    const double *ina[3];
    for (int a = 0; a < plan.nA; ++a) ina[a] = TA[a];
    if (plan.nB > 0)
      launch_band_pass_multi(ina, plan.nA, TB, plan.B_in, plan.B_ord, plan.nB, 1, n, n, n3, band,
                             s, R);
    for (int q = 0; q < plan.nB; ++q) ins[q] = plain_ptr<const double>(TB[q]);
  }
}

// w = A z followed by CGS2 pass 1 (h1 = V^T w) of an Arnoldi step: for collocation the
// operator's last pass and pass 1 run as one kernel (one launch and one read of w fewer).
template <class Tin>
void Ctx::operator_and_pass1(IdxPtr<const Tin> in, int R, cudaStream_t s) {
  if (scheme == 1 || !fuse_pass1()) {
    apply_operator<Tin>(in, w.ptr, R, s);
    launch_cgs2_coeffs(ws, w.ptr, s);
    return;
  }
  IdxPtr<const double> ins[6];
  operator_passes<Tin>(in, R, s, ins);
  launch_cgs_pass1_op(ws, make_contract_args<double>(ins, plan.terms, plan.nterm), band, n,
                      w.ptr, s);
  launch_cgs2_pass2(ws, w.ptr, s);
}

// Algorithmic FLOPs of one application of the operator to one vector, from the pass
// plan: 2 per stored band entry of every banded product, 2 per contracted collocation term
// (its coefficient), 1 per quadrature point of a Q-weighted WQ term (the multiplication by
// Q_ab, on the expansion's output grid).
double Ctx::operator_flops() const {
  double fl = 0.0;
  if (scheme == 1) {
    for (const WqPass &P : wq_op) {
      const double out = (double)P.ext_out[0] * P.ext_out[1] * P.ext_out[2];
      const double in = (double)P.ext_in[0] * P.ext_in[1] * P.ext_in[2];
      const int w = P.kind == 0 ? fac->W : fac->WW;
      for (int t = 0; t < P.nterm; ++t)
        fl += 2.0 * w * out + (P.coef[t] >= 0 ? in : 0.0) + (P.fan ? P.nfan[t] * out : 0.0);
    }
    return fl;
  }
  const int passes = plan.nA + (d == 3 ? plan.nB : 0) + plan.nterm;
  return (double)N * (2.0 * fac->W * passes + 2.0 * plan.nterm);
}

template void Ctx::apply_operator<double>(IdxPtr<const double>, double *, int, cudaStream_t);
template void Ctx::apply_operator<float>(IdxPtr<const float>, double *, int, cudaStream_t);
template void Ctx::operator_and_pass1<double>(IdxPtr<const double>, int, cudaStream_t);
template void Ctx::operator_and_pass1<float>(IdxPtr<const float>, int, cudaStream_t);

// ------------------------------------------------------------------ FD (FP64)
template <class Tout>
static void fd_chain_fp64(const Ctx &c, IdxPtr<const double> in, IdxPtr<Tout> out, int R,
                          cudaStream_t s) {
  const Factor1D &f = *c.fac;
  const int n = c.n;
  double *t0 = c.fd_scratch.ptr, *t1 = c.fd_scratch.ptr + (size_t)R * c.N;
  const int M = (int)(R * (c.N / n));
  auto P = [](double *p) { return plain_ptr<double>(p); };
  auto Pc = [](const double *p) { return plain_ptr<const double>(p); };
  if (c.fold_ok) {
    // d forward products (the last one fused with the diagonal), d inverse products,
    // each on folded vectors with half the FMAs of a dense product
    FdScale sc{nullptr, nullptr, nullptr, n, c.dinv.ptr};
    IdxPtr<const double> src = in;
    double *bufs[2] = {t0, t1};
    for (int g = 0; g < 2 * c.d; ++g) {
      const bool fwd = g < c.d, last = g == 2 * c.d - 1;
      const double *B = fwd ? f.d_Bf.ptr : f.d_Bi.ptr;
      const FdScale *scp = (g == c.d - 1) ? &sc : nullptr;
      if constexpr (std::is_same_v<Tout, double>) {
        if (use_fold_fma(M, n)) {
          launch_gemm_fp64_fold_fma(fwd ? 0 : 1, src, fwd ? f.d_BfT.ptr : f.d_BiT.ptr,
                                    last ? out : P(bufs[g & 1]), M, n, f.ne,
                                    scp ? c.dinv.ptr : nullptr, s, R);
          src = Pc(bufs[g & 1]);
          continue;
        }
      }
      if (last) {
        launch_gemm_fp64_fold<Tout>(1, src, B, out, M, n, f.ne, nullptr, s, R);
      } else {
        launch_gemm_fp64_fold<double>(fwd ? 0 : 1, src, B, P(bufs[g & 1]), M, n, f.ne, scp, s, R);
        src = Pc(bufs[g & 1]);
      }
    }
    return;
  }
  // dense products: the g-th forward (inverse) product contracts direction g with that
  // direction's V^T (U); the diagonal (dinv, each direction's eigenvalues) is fused into
  // the d-th forward product
  const Factor1D &f0 = *c.facd[0], &f1 = *c.facd[1], &f2 = *c.facd[2];
  if (c.d == 2) {
    FdScale sc{f0.d_lam.ptr, nullptr, f1.d_lam.ptr, n, c.dinv.ptr};
    launch_gemm_fp64_dense_mma<double>(in, f0.d_Vt.ptr, P(t0), M, n, nullptr, s, R);
    launch_gemm_fp64_dense_mma<double>(Pc(t0), f1.d_Vt.ptr, P(t1), M, n, &sc, s, R);
    launch_gemm_fp64_dense_mma<double>(Pc(t1), f0.d_U.ptr, P(t0), M, n, nullptr, s, R);
    launch_gemm_fp64_dense_mma<Tout>(Pc(t0), f1.d_U.ptr, out, M, n, nullptr, s, R);
  } else {
    FdScale sc{f0.d_lam.ptr, f1.d_lam.ptr, f2.d_lam.ptr, n, c.dinv.ptr};
    launch_gemm_fp64_dense_mma<double>(in, f0.d_Vt.ptr, P(t0), M, n, nullptr, s, R);
    launch_gemm_fp64_dense_mma<double>(Pc(t0), f1.d_Vt.ptr, P(t1), M, n, nullptr, s, R);
    launch_gemm_fp64_dense_mma<double>(Pc(t1), f2.d_Vt.ptr, P(t0), M, n, &sc, s, R);
    launch_gemm_fp64_dense_mma<double>(Pc(t0), f0.d_U.ptr, P(t1), M, n, nullptr, s, R);
    launch_gemm_fp64_dense_mma<double>(Pc(t1), f1.d_U.ptr, P(t0), M, n, nullptr, s, R);
    launch_gemm_fp64_dense_mma<Tout>(Pc(t0), f2.d_U.ptr, out, M, n, nullptr, s, R);
  }
}

void Ctx::precond(IdxPtr<const double> in, double *out, int R, cudaStream_t s) {
  ensure_capacity(R);
  if (prec == IGA_PREC_NONE) {
    throw Error{IGA_ERR_INVALID_ARG, "precond on an unpreconditioned handle"};
  } else if (prec == IGA_PREC_FP64) {
    fd_chain_fp64<double>(*this, in, plain_ptr<double>(out), R, s);
  } else if (prec == IGA_PREC_FP64_TC) {
    if (!f64tc) throw Error{IGA_ERR_CUDA, "FP64 tensor-core FD context missing"};
    f64tc_fd_apply(*f64tc, in, plain_ptr<double>(out), R, s);
  } else {
    if (!tc) throw Error{IGA_ERR_CUDA, "tensor-core FD context missing"};
    tc_fd_apply_f64out(*tc, in, out, R, s);
  }
}

// ------------------------------------------------------------------ Krylov workspace
void Ctx::ensure_ws(int max_iter, int R) {
  ensure_capacity(R);
  if (max_iter <= ws_max_iter && R <= ws_R) {
    ws.R = R;
    return;
  }
  if (pending) throw Error{IGA_ERR_INVALID_ARG, "a solve is in flight on this handle"};
  drop_graphs();
  const int mi = std::max(max_iter, ws_max_iter);
  const int Rc = std::max(R_max, std::max(R, ws_R));
  const int nblk = reduce_blocks(N, grid_mode);
  const size_t vecs = (size_t)Rc * N;
  V.alloc((size_t)(mi + 1) * vecs);
  IGA_CUDA_TRY(cudaMemsetAsync(V.ptr, 0, (size_t)(mi + 1) * vecs * 8, stream));
  if (prec == IGA_PREC_FP64 || prec == IGA_PREC_FP64_TC) Zd.alloc((size_t)mi * vecs);
  if (tensor_core_prec(prec)) Zf.alloc((size_t)mi * vecs);
  const long long hstride = (long long)(mi + 1) * mi;
  H.alloc((size_t)Rc * hstride);
  cs.alloc((size_t)Rc * (mi + 1));
  sn.alloc((size_t)Rc * (mi + 1));
  g.alloc((size_t)Rc * (mi + 2));
  y.alloc((size_t)Rc * (mi + 2));
  hist.alloc((size_t)Rc * (mi + 2));
  const long long pstride = (long long)nblk * (mi + 2);
  partials.alloc((size_t)Rc * pstride);
  scal.alloc((size_t)8 * Rc);
  counter.alloc(Rc);
  st.alloc(1);
  rs.alloc(Rc);
  IGA_CUDA_TRY(cudaMemsetAsync(counter.ptr, 0, Rc * sizeof(unsigned int), stream));
  IGA_CUDA_TRY(cudaMemsetAsync(H.ptr, 0, (size_t)Rc * hstride * 8, stream));
  IGA_CUDA_TRY(cudaMemsetAsync(hist.ptr, 0, (size_t)Rc * (mi + 2) * 8, stream));
  if (h_st) cudaFreeHost(h_st);
  if (h_rs) cudaFreeHost(h_rs);
  if (h_hist) cudaFreeHost(h_hist);
  h_st = nullptr;
  h_rs = nullptr;
  h_hist = nullptr;
  IGA_CUDA_TRY(cudaMallocHost(&h_st, sizeof(SolveState)));
  IGA_CUDA_TRY(cudaMallocHost(&h_rs, Rc * sizeof(RhsState)));
  IGA_CUDA_TRY(cudaMallocHost(&h_hist, (size_t)Rc * (mi + 2) * 8));
  ws = KrylovWs{};
  ws.V = V.ptr;
  if (prec == IGA_PREC_FP64 || prec == IGA_PREC_FP64_TC) {
    ws.Z = Zd.ptr;
    ws.z_fp32 = 0;
  } else if (prec == IGA_PREC_NONE) {
    ws.Z = V.ptr;  // P = I: z_k = v_k
    ws.z_fp32 = 0;
  } else {
    ws.Z = Zf.ptr;
    ws.z_fp32 = 1;
  }
  ws.H = H.ptr;
  ws.hstride = hstride;
  ws.cs = cs.ptr;
  ws.sn = sn.ptr;
  ws.g = g.ptr;
  ws.y = y.ptr;
  ws.hist = hist.ptr;
  ws.partials = partials.ptr;
  ws.pstride = pstride;
  ws.counter = counter.ptr;
  ws.scal = scal.ptr;
  ws.st = st.ptr;
  ws.rs = rs.ptr;
  ws.nblk = nblk;
  ws.N = N;
  ws.max_iter = mi;
  ws.R = R;
  ws_max_iter = mi;
  ws_R = Rc;
}

// ------------------------------------------------------------------ GMRES steps
// (ws.R is the number of right-hand sides of the graph being built or run)
void Ctx::launch_iteration(cudaGraphConditionalHandle cond, int has_cond, cudaStream_t s) {
  const int R = ws.R;
  const long long blk = (long long)R * N;
  const int *kptr = &ws.st->k;
  IdxPtr<const double> vk{ws.V, kptr, 0, blk};
  if (prec == IGA_PREC_NONE) {
    operator_and_pass1<double>(vk, R, s);
  } else if (prec == IGA_PREC_FP64) {
    IdxPtr<double> zk{(double *)ws.Z, kptr, 0, blk};
    fd_chain_fp64<double>(*this, vk, zk, R, s);
    operator_and_pass1<double>(IdxPtr<const double>{(const double *)ws.Z, kptr, 0, blk}, R, s);
  } else if (prec == IGA_PREC_FP64_TC) {
    if (!f64tc) throw Error{IGA_ERR_CUDA, "FP64 tensor-core FD context missing"};
    IdxPtr<double> zk{(double *)ws.Z, kptr, 0, blk};
    f64tc_fd_apply(*f64tc, vk, zk, R, s);
    operator_and_pass1<double>(IdxPtr<const double>{(const double *)ws.Z, kptr, 0, blk}, R, s);
  } else {
    if (!tc) throw Error{IGA_ERR_CUDA, "tensor-core FD context missing"};
    IdxPtr<float> zk{(float *)ws.Z, kptr, 0, blk};
    tc_fd_apply(*tc, vk, zk, R, s);
    operator_and_pass1<float>(IdxPtr<const float>{(const float *)ws.Z, kptr, 0, blk}, R, s);
  }
  // the Givens update of column k needs only passes 1 and 2: it runs on a side stream
  // beside pass 3, and the step ends when both have finished
  IGA_CUDA_TRY(cudaEventRecord(fork_ev, s));
  IGA_CUDA_TRY(cudaStreamWaitEvent(side_stream, fork_ev, 0));
  launch_givens(ws, cond, has_cond, side_stream);
  launch_cgs2_vector(ws, w.ptr, s);
  IGA_CUDA_TRY(cudaEventRecord(join_ev, side_stream));
  IGA_CUDA_TRY(cudaStreamWaitEvent(s, join_ev, 0));
}

void Ctx::launch_solve_prologue(int use_x0, cudaGraphConditionalHandle cond, int has_cond,
                                cudaStream_t s) {
  const int R = ws.R;
  const double *r0 = b.ptr;
  if (use_x0) {
    apply_operator<double>(plain_ptr<const double>(x0.ptr), w.ptr, R, s);
    launch_axpby(b.ptr, w.ptr, 1.0, -1.0, r.ptr, (long long)R * N, s);
    r0 = r.ptr;
  }
  launch_init_solve(ws, b.ptr, r0, cond, has_cond, s);
}

void Ctx::launch_solve_epilogue(int use_x0, cudaStream_t s) {
  const int R = ws.R;
  launch_finish(ws, x0.ptr, use_x0, x.ptr, s);
  apply_operator<double>(plain_ptr<const double>(x.ptr), w.ptr, R, s);
  launch_residual_norm(ws, b.ptr, w.ptr, r.ptr, s);
}

SolveGraph &Ctx::graph_for(int R, int use_x0) {
  const auto key = std::make_pair(R, use_x0);
  auto it = graphs.find(key);
  if (it != graphs.end()) return it->second;
  const double tw = wall_seconds();
  std::unique_lock<DeviceLock> dlk(device_mutex());
  const double tl = wall_seconds();
  ws.R = R;
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
    cudaGraphDestroy(sg.graph);
    throw;
  }
  IGA_CUDA_TRY(cudaStreamEndCapture(s, &sg.graph));
  const long long c1 = g_launch_count;
  IGA_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
  try {
    launch_iteration(cond, 1, s);
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
  if (verbose_level() >= 2)
    std::fprintf(stderr, "iga solve graph d=%d n=%d R=%d: lock wait %.1f ms, capture and "
                 "instantiation %.1f ms\n", d, n, R, 1e3 * (tl - tw), 1e3 * (wall_seconds() - tl));
  return graphs[key] = sg;
}

static bool eager_mode() {
  const char *e = std::getenv("IGA_EAGER");
  return e && e[0] == '1';
}

void Ctx::enqueue(int R, const double *rhs_dev, double *x_dev, int use_x0, double tol,
                  int max_iter) {
  if (pending) throw Error{IGA_ERR_INVALID_ARG, "a solve is already in flight on this handle"};
  ensure_ws(max_iter, R);
  SolveState hs{};
  hs.tol = tol;
  hs.max_iter = max_iter;
  hs.R = R;
  *h_st = hs;
  const size_t bytes = (size_t)R * N * 8;
  IGA_CUDA_TRY(cudaMemcpyAsync(ws.st, h_st, sizeof(SolveState), cudaMemcpyHostToDevice, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(b.ptr, rhs_dev, bytes, cudaMemcpyDeviceToDevice, stream));
  if (use_x0)
    IGA_CUDA_TRY(cudaMemcpyAsync(x0.ptr, x_dev, bytes, cudaMemcpyDeviceToDevice, stream));
  if (!eager_mode()) {
    SolveGraph &sg = graph_for(R, use_x0);
    IGA_CUDA_TRY(cudaGraphLaunch(sg.exec, stream));
  } else {
    ws.R = R;
    launch_solve_prologue(use_x0, 0, 0, stream);
    for (int it = 0; it <= max_iter; ++it) {
      IGA_CUDA_TRY(cudaMemcpyAsync(h_st, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, stream));
      IGA_CUDA_TRY(cudaStreamSynchronize(stream));
      if (h_st->active == 0) break;
      launch_iteration(0, 0, stream);
    }
    launch_solve_epilogue(use_x0, stream);
  }
  IGA_CUDA_TRY(cudaMemcpyAsync(x_dev, x.ptr, bytes, cudaMemcpyDeviceToDevice, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(h_st, ws.st, sizeof(SolveState), cudaMemcpyDeviceToHost, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(h_rs, ws.rs, R * sizeof(RhsState), cudaMemcpyDeviceToHost, stream));
  IGA_CUDA_TRY(cudaMemcpyAsync(h_hist, ws.hist, (size_t)R * (ws_max_iter + 2) * 8,
                               cudaMemcpyDeviceToHost, stream));
  IGA_CUDA_TRY(cudaEventRecord(done_ev, stream));
  pending = true;
  pend_R = R;
  pend_max_iter = max_iter;
  pend_tol = tol;
}

bool Ctx::ready() {
  if (!pending) return true;
  const cudaError_t e = cudaEventQuery(done_ev);
  if (e == cudaSuccess) return true;
  if (e == cudaErrorNotReady) return false;
  IGA_CUDA_TRY(e);
  return false;
}

// Per right-hand side: iters[r], hist_out[r*(max_iter+1) + j], relres[r], status_out[r].
iga_status Ctx::collect(int *iters, double *hist_out, double *relres, int *status_out) {
  if (!pending) throw Error{IGA_ERR_INVALID_ARG, "no solve in flight on this handle"};
  pending = false;
  IGA_CUDA_TRY(cudaEventSynchronize(done_ev));
  int *ew = tc ? tc_fd_error_word(*tc) : f64tc ? f64tc_error_word(*f64tc) : nullptr;
  if (ew) {
    int err = 0;
    IGA_CUDA_TRY(cudaMemcpy(&err, ew, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
      IGA_CUDA_TRY(cudaMemset(ew, 0, sizeof(int)));
      throw Error{IGA_ERR_DEVICE_TIMEOUT,
                  "a tensor-core FD wait timed out (code " + std::to_string(err) + ")"};
    }
  }
  const int R = pend_R, mi = pend_max_iter;
  iga_status overall = IGA_OK;
  for (int q = 0; q < R; ++q) {
    const RhsState &s = h_rs[q];
    if (iters) iters[q] = s.kconv;
    if (hist_out) {
      const double *h = h_hist + (size_t)q * (ws_max_iter + 2);
      double *o = hist_out + (size_t)q * (mi + 1);
      for (int j = 0; j <= mi; ++j) o[j] = j <= s.kconv ? h[j] : 0.0;
    }
    if (relres) relres[q] = s.relres_true;
    iga_status st_q = IGA_OK;
    if (s.flag == 4 || !std::isfinite(s.relres_true)) st_q = IGA_ERR_NAN;
    else if (s.flag == 2 && pend_tol > 0.0) st_q = IGA_ERR_NO_CONVERGENCE;
    if (status_out) status_out[q] = st_q;
    if (st_q == IGA_ERR_NAN) overall = IGA_ERR_NAN;
    else if (st_q != IGA_OK && overall == IGA_OK) overall = st_q;
  }
  return overall;
}

// ------------------------------------------------------------------ points (host)
void Ctx::collocation_points(double *xyz) const {
  if (scheme != 0)
    throw Error{IGA_ERR_UNSUPPORTED, "collocation points of a weighted-quadrature problem: use "
                                     "iga_quadrature_points"};
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
          const double rr = r0 + (r1 - r0) * xi;
          const double X = rr * std::cos(w_ * eta), Y = rr * std::sin(w_ * eta);
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
