// Classical optimiser of the QVA workflow (Sec. 4): the paper minimises f(theta) with SciPy's BFGS
// on the host while the simulator evaluates f and its gradient. Here the same loop runs in C on
// the host around qvs_gradient (device objective + adjoint gradient per evaluation):
//   * direction d = -H g, H the inverse-Hessian estimate (H_0 = I; reset to I when d is not a
//     descent direction);
//   * backtracking line search from step 1, halving until f(x + a d) <= f(x) + c1 a g.d
//     (c1 = 1e-4), at most kMaxHalvings times;
//   * with s = x_new - x, y = g_new - g: H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T,
//     rho = 1 / y.s, skipped when y.s <= 0;
//   * stop when max |g| <= gtol (stop 0), after max_iter iterations (stop 1), or when no step of
//     the line search decreases f enough (stop 2: rounding of the objective hides any further
//     descent; x, f and g stay at the last accepted point, as SciPy's BFGS ends on precision loss).
#include <math.h>

#include <vector>

#include "qvs_internal.h"

static const int kMaxHalvings = 30;

static int qvs_bfgs_minimize_impl(int n, double* x, qvs_fg_fn fg, void* user, double gtol, int max_iter,
                                  double* f_out, int* iters_out, int* evals_out, int* stop_out) {
  if (n < 1 || n > 8192 || !x || !fg || max_iter < 0 || !(gtol >= 0.0)) return QVS_EINVAL;
  const size_t N = (size_t)n;
  std::vector<double> H(N * N, 0.0), g(N), gn(N), xn(N), d(N), s(N), y(N), Hy(N);
  auto reset = [&]() {
    for (size_t i = 0; i < N * N; ++i) H[i] = 0.0;
    for (size_t i = 0; i < N; ++i) H[i * N + i] = 1.0;
  };
  reset();
  double f = 0.0;
  QVS_TRY(fg(x, &f, g.data(), user));
  int evals = 1, it = 0;
  auto gmax = [&](const std::vector<double>& v) {
    double m = 0.0;
    for (double e : v) m = fmax(m, fabs(e));
    return m;
  };
  int stop = 1;
  while (it < max_iter) {
    if (gmax(g) <= gtol) {
      stop = 0;
      break;
    }
    for (size_t i = 0; i < N; ++i) {
      double acc = 0.0;
      for (size_t j = 0; j < N; ++j) acc += H[i * N + j] * g[j];
      d[i] = -acc;
    }
    double slope = 0.0;
    for (size_t i = 0; i < N; ++i) slope += g[i] * d[i];
    if (slope >= 0.0) {
      reset();
      slope = 0.0;
      for (size_t i = 0; i < N; ++i) {
        d[i] = -g[i];
        slope += g[i] * d[i];
      }
    }
    double a = 1.0, fn = 0.0;
    bool accepted = false;
    for (int halving = 0; halving <= kMaxHalvings; ++halving) {
      for (size_t i = 0; i < N; ++i) xn[i] = x[i] + a * d[i];
      QVS_TRY(fg(xn.data(), &fn, gn.data(), user));
      ++evals;
      if (fn <= f + 1e-4 * a * slope) {
        accepted = true;
        break;
      }
      a *= 0.5;
    }
    if (!accepted) {
      stop = 2;
      break;
    }
    double ys = 0.0;
    for (size_t i = 0; i < N; ++i) {
      s[i] = xn[i] - x[i];
      y[i] = gn[i] - g[i];
      ys += y[i] * s[i];
    }
    if (ys > 0.0) {
      // H <- H - rho (s (H y)^T + (H y) s^T) + (rho^2 y.Hy + rho) s s^T   (the product form expanded;
      // H is symmetric, so y^T H = (H y)^T)
      const double rho = 1.0 / ys;
      double yHy = 0.0;
      for (size_t i = 0; i < N; ++i) {
        double acc = 0.0;
        for (size_t j = 0; j < N; ++j) acc += H[i * N + j] * y[j];
        Hy[i] = acc;
      }
      for (size_t i = 0; i < N; ++i) yHy += y[i] * Hy[i];
      const double cs = rho * rho * yHy + rho;
      for (size_t i = 0; i < N; ++i)
        for (size_t j = 0; j < N; ++j)
          H[i * N + j] += -rho * (s[i] * Hy[j] + Hy[i] * s[j]) + cs * s[i] * s[j];
    }
    for (size_t i = 0; i < N; ++i) {
      x[i] = xn[i];
      g[i] = gn[i];
    }
    f = fn;
    ++it;
  }
  if (stop == 1 && gmax(g) <= gtol) stop = 0;
  if (f_out) *f_out = f;
  if (iters_out) *iters_out = it;
  if (evals_out) *evals_out = evals;
  if (stop_out) *stop_out = stop;
  return QVS_OK;
}

extern "C" int qvs_bfgs_minimize(int n, double* x, qvs_fg_fn fg, void* user, double gtol, int max_iter,
                                 double* f_out, int* iters_out, int* evals_out, int* stop_out) {
  return qvs::guarded([&] {
    return qvs_bfgs_minimize_impl(n, x, fg, user, gtol, max_iter, f_out, iters_out, evals_out, stop_out);
  });
}

namespace {
struct OptCtx {
  qvs_t h;
  int p;
  std::vector<double> gs, ts, dg, dt;
};
// theta = (gamma_1, t_1, gamma_2, t_2, ...) (the layer order of Example 1)
int qva_fg(const double* th, double* f, double* g, void* user) {
  OptCtx* c = static_cast<OptCtx*>(user);
  for (int k = 0; k < c->p; ++k) {
    c->gs[k] = th[2 * k];
    c->ts[k] = th[2 * k + 1];
  }
  QVS_TRY(qvs_gradient(c->h, c->p, c->gs.data(), c->ts.data(), f, c->dg.data(), c->dt.data()));
  for (int k = 0; k < c->p; ++k) {
    g[2 * k] = c->dg[k];
    g[2 * k + 1] = c->dt[k];
  }
  return QVS_OK;
}
}  // namespace

static int qvs_optimise_impl(qvs_t h, int p, double* gammas, double* ts, double gtol, int max_iter, double* f_out,
                             int* iters_out, int* evals_out, int* stop_out) {
  if (!h || p < 1 || p > 4096 || !gammas || !ts) return QVS_EINVAL;
  OptCtx c{h, p, std::vector<double>(p), std::vector<double>(p), std::vector<double>(p), std::vector<double>(p)};
  std::vector<double> th(2 * (size_t)p);
  for (int k = 0; k < p; ++k) {
    th[2 * k] = gammas[k];
    th[2 * k + 1] = ts[k];
  }
  QVS_TRY(qvs_bfgs_minimize(2 * p, th.data(), qva_fg, &c, gtol, max_iter, f_out, iters_out, evals_out, stop_out));
  for (int k = 0; k < p; ++k) {
    gammas[k] = th[2 * k];
    ts[k] = th[2 * k + 1];
  }
  return QVS_OK;
}

extern "C" int qvs_optimise(qvs_t h, int p, double* gammas, double* ts, double gtol, int max_iter, double* f_out,
                            int* iters_out, int* evals_out, int* stop_out) {
  return qvs::guarded([&] {
    return qvs_optimise_impl(h, p, gammas, ts, gtol, max_iter, f_out, iters_out, evals_out, stop_out);
  });
}
