// fit.cpp -- identification of theta by maximising the likelihood (Sec. 5,
// App. B): the simplex method of Nelder and Mead over (nu, ell, sigma2) on one
// tree, every evaluation a full H-likelihood on the device (hlc_loglik).
//
// The simplex method is written from its published definition (J. A. Nelder,
// R. Mead, Comput. J. 7 (1965) 308-313, in the form of Lagarias, Reeds,
// Wright, Wright, SIAM J. Optim. 9 (1998) 112-147) with the standard
// coefficients: reflection 1, expansion 2, contraction 1/2, shrink 1/2.
// One iteration is one of: accept the reflected point, accept the expanded
// point, accept an outside or inside contraction, or shrink towards the best
// vertex.  The simplex starts from x0 and the vertices x0 + step_i e_i; the
// iteration stops when the simplex size -- the root mean square distance of
// its vertices from their centroid -- falls below size_tol, or after
// max_iter iterations.  The App. B listing sets the steps to 0.02, 0.04 and
// 0.01 for (nu, ell, sigma2), the size tolerance to 1e-5 and the iteration
// limit to 200, and minimises -L.

#include <math.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/hlc.h"

namespace {

struct Vertex {
  std::vector<double> x;
  double f;
};

double simplex_size(const std::vector<Vertex>& S) {
  const size_t d = S[0].x.size();
  std::vector<double> c(d, 0.0);
  for (const Vertex& v : S)
    for (size_t i = 0; i < d; ++i) c[i] += v.x[i];
  for (size_t i = 0; i < d; ++i) c[i] /= (double)S.size();
  double s = 0.0;
  for (const Vertex& v : S)
    for (size_t i = 0; i < d; ++i) s += (v.x[i] - c[i]) * (v.x[i] - c[i]);
  return sqrt(s / (double)S.size());
}

// f values that are NaN count as +inf (a failed evaluation loses every
// comparison)
double clean(double f) { return f == f ? f : INFINITY; }

}  // namespace

extern "C" {

int hlc_nelder_mead(int dim, double* x, const double* step, double size_tol, int max_iter, hlc_objective f,
                    void* user, double* fmin, int* iters) {
  if (dim < 1 || dim > 64 || !x || !step || !f || max_iter < 0 || !(size_tol >= 0.0)) return HLC_ERR_ARG;
  const size_t d = (size_t)dim;
  std::vector<Vertex> S(d + 1);
  S[0].x.assign(x, x + d);
  S[0].f = clean(f(S[0].x.data(), user));
  for (size_t i = 0; i < d; ++i) {
    S[i + 1].x = S[0].x;
    S[i + 1].x[i] += step[i];
    S[i + 1].f = clean(f(S[i + 1].x.data(), user));
  }
  // order by f; ties keep the earlier vertex first
  auto order = [&]() {
    std::stable_sort(S.begin(), S.end(), [](const Vertex& a, const Vertex& b) { return a.f < b.f; });
  };
  std::vector<double> c(d), xr(d), xe(d), xc(d);
  auto eval = [&](std::vector<double>& p) { return clean(f(p.data(), user)); };
  int it = 0;
  order();
  while (it < max_iter && simplex_size(S) >= size_tol) {
    ++it;
    // centroid of the best d vertices (summed best first)
    std::fill(c.begin(), c.end(), 0.0);
    for (size_t v = 0; v < d; ++v)
      for (size_t i = 0; i < d; ++i) c[i] += S[v].x[i];
    for (size_t i = 0; i < d; ++i) c[i] /= (double)d;
    Vertex& worst = S[d];
    for (size_t i = 0; i < d; ++i) xr[i] = c[i] + (c[i] - worst.x[i]);
    const double fr = eval(xr);
    bool shrink = false;
    if (fr < S[0].f) {
      for (size_t i = 0; i < d; ++i) xe[i] = c[i] + 2.0 * (c[i] - worst.x[i]);
      const double fe = eval(xe);
      if (fe < fr) {
        worst.x = xe;
        worst.f = fe;
      } else {
        worst.x = xr;
        worst.f = fr;
      }
    } else if (fr < S[d - 1].f) {
      worst.x = xr;
      worst.f = fr;
    } else if (fr < worst.f) {
      // outside contraction
      for (size_t i = 0; i < d; ++i) xc[i] = c[i] + 0.5 * (xr[i] - c[i]);
      const double fc = eval(xc);
      if (fc <= fr) {
        worst.x = xc;
        worst.f = fc;
      } else {
        shrink = true;
      }
    } else {
      // inside contraction
      for (size_t i = 0; i < d; ++i) xc[i] = c[i] + 0.5 * (worst.x[i] - c[i]);
      const double fc = eval(xc);
      if (fc < worst.f) {
        worst.x = xc;
        worst.f = fc;
      } else {
        shrink = true;
      }
    }
    if (shrink) {
      for (size_t v = 1; v <= d; ++v) {
        for (size_t i = 0; i < d; ++i) S[v].x[i] = S[0].x[i] + 0.5 * (S[v].x[i] - S[0].x[i]);
        S[v].f = eval(S[v].x);
      }
    }
    order();
  }
  std::copy(S[0].x.begin(), S[0].x.end(), x);
  if (fmin) *fmin = S[0].f;
  if (iters) *iters = it;
  return HLC_OK;
}

void hlc_default_fit_opts(hlc_fit_opts* o) {
  if (!o) return;
  o->step[0] = 0.02;  // nu
  o->step[1] = 0.04;  // ell
  o->step[2] = 0.01;  // sigma2
  o->size_tol = 1e-5;
  o->max_iter = 200;
  o->free_mask = 7;
}

}  // extern "C"

namespace {

struct FitState {
  hlc_ctx* ctx;
  hlc_tree* tree;
  const double* z;
  hlc_theta base;
  int mask;
  int evals = 0, failed = 0, hard_error = 0;
  double* trace;
  int trace_cap;
  int traced = 0;
};

// the free parameters, in the order (nu, ell, sigma2) of the App. B listing
void unpack(const FitState& S, const double* x, hlc_theta* th) {
  *th = S.base;
  int q = 0;
  if (S.mask & 1) th->nu = x[q++];
  if (S.mask & 2) th->ell = x[q++];
  if (S.mask & 4) th->sigma2 = x[q++];
}

double neg_loglik(const double* x, void* user) {
  FitState& S = *static_cast<FitState*>(user);
  hlc_theta th;
  unpack(S, x, &th);
  S.evals += 1;
  if (!(th.nu > 0.0 && th.ell > 0.0 && th.sigma2 > 0.0 && th.nu < 20.0)) {
    S.failed += 1;
    return INFINITY;  // outside the parameter domain
  }
  hlc_result r;
  const int st = hlc_loglik(S.ctx, S.tree, &th, S.z, &r);
  double v = INFINITY;
  if (st == HLC_OK) {
    v = -r.loglik;
  } else if (st == HLC_ERR_NOT_SPD || st == HLC_ERR_NUMERIC || st == HLC_ERR_RANK) {
    S.failed += 1;  // this theta cannot be evaluated: the simplex moves away
  } else {
    S.hard_error = st;  // device or state failure: stop as soon as possible
  }
  if (S.trace && S.traced < S.trace_cap) {
    double* t = S.trace + 5 * (int64_t)S.traced;
    t[0] = th.nu;
    t[1] = th.ell;
    t[2] = th.sigma2;
    t[3] = -v;
    t[4] = (double)st;
    S.traced += 1;
  }
  return v;
}

}  // namespace

extern "C" int hlc_fit(hlc_ctx* ctx, hlc_tree* t, const double* z, const hlc_theta* start, const hlc_fit_opts* opts,
                       double* trace, int trace_cap, hlc_fit_result* out) {
  if (!ctx || !t || !z || !start || !out || (trace_cap > 0 && !trace)) return HLC_ERR_ARG;
  hlc_fit_opts o;
  if (opts)
    o = *opts;
  else
    hlc_default_fit_opts(&o);
  if ((o.free_mask & 7) == 0 || (o.free_mask & ~7) || o.max_iter < 0) return HLC_ERR_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  FitState S{ctx, t, z, *start, o.free_mask};
  S.trace = trace_cap > 0 ? trace : nullptr;
  S.trace_cap = trace_cap;
  double x[3], step[3];
  int d = 0;
  const double x0[3] = {start->nu, start->ell, start->sigma2};
  for (int i = 0; i < 3; ++i)
    if (o.free_mask & (1 << i)) {
      x[d] = x0[i];
      step[d] = o.step[i];
      ++d;
    }
  double fbest = INFINITY;
  int it = 0;
  // a device or state failure inside an evaluation ends the fit: the
  // objective then returns +inf for every later point, which the simplex
  // cannot improve on, so it collapses without further device work
  auto guarded = [](const double* xx, void* u) -> double {
    FitState& s = *static_cast<FitState*>(u);
    if (s.hard_error) return INFINITY;
    return neg_loglik(xx, u);
  };
  int st = hlc_nelder_mead(d, x, step, o.size_tol, o.max_iter, guarded, &S, &fbest, &it);
  if (st) return st;
  if (S.hard_error) return S.hard_error;
  std::memset(out, 0, sizeof(*out));
  unpack(S, x, &out->theta);
  out->loglik = -fbest;
  out->iterations = it;
  out->evaluations = S.evals;
  out->failed_evals = S.failed;
  out->traced = S.traced;
  out->converged = it < o.max_iter ? 1 : 0;
  out->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (!(fbest < INFINITY)) return HLC_ERR_NUMERIC;  // no evaluation succeeded
  return HLC_OK;
}
