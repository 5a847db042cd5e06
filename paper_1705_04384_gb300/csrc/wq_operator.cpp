// Weighted-quadrature Galerkin problems (Sec. 2.3): setup of the coefficient fields on
// the quadrature grid, the plan of the matrix-free operator A_wq (eq. WQapprox) as a chain
// of banded passes, its execution, the load vector and the quadrature points.
//
// A_wq u = sum over active terms (a, b) of W_ab diag(Q_ab) B_b u with B_b = (x)_l B^{(b_l)}
// and W_ab = (x)_l W^{(a_l, b_l)} (a_l = [l == a], b_l = [l == b]).  The expansion half is a
// tree over the directions d-1 .. 0 (intermediates identified by the derivative orders of
// the directions already expanded, so shared prefixes are computed once); the contraction
// half runs over the directions 0 .. d-1, multiplying by Q_ab in the first pass and adding
// the terms whose remaining rules coincide.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "context.h"

namespace iga {

// field index of Q_ab: 2D (11, 22, 12), 3D (11, 22, 33, 12, 13, 23); the last is |det J|
static int wq_field(int d, int a, int b) {
  if (a == b) return a;
  const int lo = std::min(a, b), hi = std::max(a, b);
  if (d == 2) return 2;
  return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}

void Ctx::setup_wq() {
  nq = fac->nq;
  Nq = 1;
  for (int l = 0; l < d; ++l) Nq *= nq;
  wq_nf = d == 2 ? 4 : 7;
  ldq = (Nq + 31) / 32 * 32;
  wq_fields.alloc((size_t)wq_nf * ldq);
  const double *xq = fac->d_xq.ptr;
  launch_wq_fields(d, geom, xq, xq, xq, nq, nq, d == 3 ? nq : 1, wq_fields.ptr, ldq, stream);
  DevBuf<unsigned long long> dmax;
  dmax.alloc(wq_nf);
  launch_field_maxabs(wq_fields.ptr, ldq, Nq, wq_nf, dmax.ptr, stream);
  unsigned long long hmax[7];
  IGA_CUDA_TRY(cudaMemcpyAsync(hmax, dmax.ptr, wq_nf * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, stream));
  IGA_CUDA_TRY(cudaStreamSynchronize(stream));
  double mx[7], scale = 0.0;
  for (int f = 0; f < wq_nf; ++f) {
    std::memcpy(&mx[f], &hmax[f], sizeof(double));
    if (!std::isfinite(mx[f])) throw Error{IGA_ERR_INVALID_ARG, "geometry map is singular"};
    if (f < d) scale = std::max(scale, mx[f]);
  }
  // a coefficient that vanishes identically up to rounding (the off-diagonal Q_ab of the
  // ring) contributes nothing: its terms are dropped from the plan
  for (int f = 0; f < wq_nf; ++f) wq_active[f] = mx[f] > 1e-12 * scale;
  build_wq_plan();
}

void Ctx::build_wq_plan() {
  wq_op.clear();
  wq_load.clear();
  wq_slot_size.clear();
  auto new_slot = [&](const int *ext) {
    wq_slot_size.push_back((long long)ext[0] * ext[1] * ext[2]);
    return (int)wq_slot_size.size() - 1;
  };
  // active terms (a, b)
  std::vector<std::pair<int, int>> terms;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b)
      if (wq_active[wq_field(d, a, b)]) terms.push_back({a, b});
  if (terms.empty()) throw Error{IGA_ERR_INVALID_ARG, "weighted quadrature: no active term"};

  // ---- expansion: directions d-1 .. 0; an intermediate after expanding directions
  // k .. d-1 is identified by its derivative orders (b_k .. b_{d-1}), packed in bits
  std::vector<int> betas;
  for (auto &t : terms)
    if (std::find(betas.begin(), betas.end(), t.second) == betas.end()) betas.push_back(t.second);
  std::map<int, int> cur;  // suffix code -> slot
  cur[0] = -1;             // before any pass: the input vector
  int ext[3] = {1, 1, 1};
  for (int l = 0; l < d; ++l) ext[l] = n;
  auto suffix = [&](int beta, int k) {  // orders of directions k .. d-1 of e_beta, as bits
    int code = 0;
    for (int l = k; l < d; ++l) code |= (l == beta ? 1 : 0) << l;
    return code;
  };
  // the last pass (direction 0) fans out: d_beta u on the quadrature grid is summed once and
  // written as Q_{a,beta} d_beta u for every active a (slot fan_slot[a][beta])
  int fan_slot[3][3];
  for (int dir = d - 1; dir >= 0; --dir) {
    WqPass P;
    P.dir = dir;
    P.kind = 0;
    P.fan = dir == 0 ? 1 : 0;
    std::memcpy(P.ext_in, ext, sizeof(ext));
    ext[dir] = nq;
    std::memcpy(P.ext_out, ext, sizeof(ext));
    std::map<int, int> next;
    for (int beta : betas) {
      const int code = suffix(beta, dir);
      if (next.count(code)) continue;
      const int t = P.nterm++;
      P.in_slot[t] = cur.at(suffix(beta, dir + 1));
      P.sel[t] = beta == dir ? 1 : 0;
      P.coef[t] = -1;
      if (P.fan) {
        next[code] = -1;
        for (int a = 0; a < d; ++a) {
          if (!wq_active[wq_field(d, a, beta)]) continue;
          const int k = P.nfan[t]++;
          P.fcoef[t][k] = wq_field(d, a, beta);
          P.fslot[t][k] = fan_slot[a][beta] = new_slot(P.ext_out);
        }
      } else {
        const int q = P.nout++;
        next[code] = q;
        P.out_of[t] = q;
      }
    }
    if (!P.fan)
      for (auto &kv : next) {
        const int q = kv.second;
        P.out_slot[q] = new_slot(P.ext_out);
        kv.second = P.out_slot[q];
      }
    cur = next;
    wq_op.push_back(P);
  }
  // Q_ab d_b u on the quadrature grid: slot fan_slot[a][b]

  // ---- contraction: directions 0 .. d-1; an item after contracting directions 0 .. k-1 is
  // identified by its remaining rules (r_k .. r_{d-1}), r_l = 2 a_l + b_l, in base-4 digits
  auto rules = [&](int a, int b) {
    int code = 0, mul = 1;
    for (int l = 0; l < d; ++l, mul *= 4) code += (2 * (l == a) + (l == b)) * mul;
    return code;
  };
  struct Item {
    int slot, code, field;
  };
  std::vector<Item> items;
  for (auto &t : terms)  // Q is already applied: no coefficient in the contraction
    items.push_back({fan_slot[t.first][t.second], rules(t.first, t.second), -1});
  auto contract_chain = [&](std::vector<Item> its, std::vector<WqPass> &chain) {
    int e[3] = {1, 1, 1};
    for (int l = 0; l < d; ++l) e[l] = nq;
    for (int dir = 0; dir < d; ++dir) {
      WqPass P;
      P.dir = dir;
      P.kind = 1;
      std::memcpy(P.ext_in, e, sizeof(e));
      e[dir] = n;
      std::memcpy(P.ext_out, e, sizeof(e));
      std::map<int, int> group;  // remaining code -> output index
      std::vector<Item> next;
      for (const Item &it : its) {
        const int rest = it.code / 4, r = it.code % 4;
        auto g = group.find(rest);
        int q;
        if (g == group.end()) {
          q = P.nout++;
          group[rest] = q;
          next.push_back({-1, rest, -1});
        } else {
          q = g->second;
        }
        if (P.nterm >= kWqMaxTerms) throw Error{IGA_ERR_INVALID_ARG, "weighted quadrature plan"};
        P.in_slot[P.nterm] = it.slot;
        P.sel[P.nterm] = r;
        P.coef[P.nterm] = it.field;
        P.out_of[P.nterm] = q;
        P.nterm++;
      }
      for (int q = 0; q < P.nout; ++q) {
        P.out_slot[q] = dir == d - 1 ? -1 : new_slot(P.ext_out);
        next[q].slot = P.out_slot[q];
      }
      // the pass kernel sums the consecutive terms of one output: group them (stable)
      int perm[kWqMaxTerms];
      for (int t = 0; t < P.nterm; ++t) perm[t] = t;
      std::stable_sort(perm, perm + P.nterm, [&](int x, int y) { return P.out_of[x] < P.out_of[y]; });
      const WqPass U = P;
      for (int t = 0; t < P.nterm; ++t) {
        P.in_slot[t] = U.in_slot[perm[t]];
        P.sel[t] = U.sel[perm[t]];
        P.coef[t] = U.coef[perm[t]];
        P.out_of[t] = U.out_of[perm[t]];
      }
      chain.push_back(P);
      its = next;
    }
  };
  contract_chain(items, wq_op);
  // load vector: the (0, 0) rule in every direction applied to |det J| g (a single term)
  contract_chain(std::vector<Item>{{-1, 0, wq_nf - 1}}, wq_load);
}

template <class Tin>
void Ctx::run_wq(const std::vector<WqPass> &chain, IdxPtr<const Tin> in, double *out, int R,
                 cudaStream_t s) {
  // slot k of R right-hand sides at R * (sizes of the slots before k)
  std::vector<long long> off(wq_slot_size.size() + 1, 0);
  for (size_t k = 0; k < wq_slot_size.size(); ++k) off[k + 1] = off[k] + wq_slot_size[k];
  const Factor1D &f = *fac;
  auto fill = [&](auto &A, const WqPass &P) {
    for (int t = 0; t < P.nterm; ++t) {
      if (P.kind == 0) {
        A.start[t] = f.d_qstart.ptr;
        A.band[t] = f.d_qband[P.sel[t]].ptr;
        A.width[t] = f.W;
      } else {
        A.start[t] = f.d_wstart.ptr;
        A.band[t] = f.d_wband[P.sel[t]].ptr;
        A.width[t] = f.WW;
      }
      A.coef[t] = P.coef[t] >= 0 ? wq_fields.ptr + P.coef[t] * ldq : nullptr;
      A.out_of[t] = P.out_of[t];
    }
    A.nterm = P.nterm;
    A.nout = P.nout;
    for (int q = 0; q < P.nout; ++q)
      A.out[q] = P.out_slot[q] < 0 ? out : wq_scratch.ptr + R * off[P.out_slot[q]];
    A.fan = P.fan;
    for (int t = 0; t < P.nterm && P.fan; ++t) {
      A.nfan[t] = P.nfan[t];
      for (int k = 0; k < P.nfan[t]; ++k) {
        A.fcoef[t][k] = wq_fields.ptr + P.fcoef[t][k] * ldq;
        A.fout[t][k] = wq_scratch.ptr + R * off[P.fslot[t][k]];
      }
    }
  };
  for (size_t k = 0; k < chain.size(); ++k) {
    const WqPass &P = chain[k];
    if (k == 0) {
      WqPassArgs<Tin> A{};
      A.vin = in;
      for (int t = 0; t < P.nterm; ++t) {
        if (P.in_slot[t] >= 0) throw Error{IGA_ERR_INVALID_ARG, "weighted quadrature plan"};
        A.in[t] = nullptr;
      }
      fill(A, P);
      launch_wq_pass<Tin>(A, P.dir, P.ext_in, P.ext_out, R, s);
    } else {
      WqPassArgs<double> A{};
      A.vin = plain_ptr<const double>(nullptr);
      for (int t = 0; t < P.nterm; ++t) {
        if (P.in_slot[t] < 0) throw Error{IGA_ERR_INVALID_ARG, "weighted quadrature plan"};
        A.in[t] = wq_scratch.ptr + R * off[P.in_slot[t]];
      }
      fill(A, P);
      launch_wq_pass<double>(A, P.dir, P.ext_in, P.ext_out, R, s);
    }
  }
}

template void Ctx::run_wq<double>(const std::vector<WqPass> &, IdxPtr<const double>, double *, int,
                                  cudaStream_t);
template void Ctx::run_wq<float>(const std::vector<WqPass> &, IdxPtr<const float>, double *, int,
                                 cudaStream_t);

void Ctx::wq_load_vector(const double *g, double *fvec, cudaStream_t s) {
  if (scheme != 1) throw Error{IGA_ERR_UNSUPPORTED, "not a weighted-quadrature problem"};
  ensure_capacity(1);
  run_wq<double>(wq_load, plain_ptr<const double>(g), fvec, 1, s);
}

// Physical quadrature points F(x_q) in the order of the quadrature grid (direction 1
// fastest), nq^d x d row-major.
void Ctx::quadrature_points(double *xyz) const {
  const std::vector<double> &x = fac->xq;
  const double r0 = geom.r_inner, r1 = geom.r_outer, w_ = 0.5 * M_PI;
  const long long n3 = d == 3 ? nq : 1;
  for (long long i3 = 0; i3 < n3; ++i3)
    for (long long i2 = 0; i2 < nq; ++i2)
      for (long long i1 = 0; i1 < nq; ++i1) {
        const long long i = i1 + nq * (i2 + nq * i3);
        const double xi = x[i1], eta = x[i2], zeta = d == 3 ? x[i3] : 0.0;
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
