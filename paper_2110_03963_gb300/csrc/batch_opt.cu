// Batched classical optimiser of the QVA workflow (Sec. 4: BFGS is the paper's default) on the
// device: every instance of a batch runs its own BFGS over theta = (gamma_1, t_1, ..., gamma_p, t_p)
// while one persistent launch evaluates the objective and adjoint gradient of all of them at once.
//
// One iteration of the loop is a CUDA graph of three steps:
//   1. the batched kernel evaluates f and grad f at every active instance's trial point
//      (instances that have stopped are skipped);
//   2. bfgs_step_kernel (one CTA per instance) advances each instance's BFGS state by one
//      evaluation: the first evaluation sets the start point; a trial point is accepted when it
//      passes the Armijo test f(x + a d) <= f(x) + c1 a g.d, then the inverse-Hessian estimate is
//      updated H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T (rho = 1/y.s, skipped when
//      y.s <= 0) and the next direction d = -H g is taken (H reset to I and d = -g when that is not
//      a descent direction); a rejected trial halves a (at most 30 times);
//   3. the number of instances still active is copied to the host, which stops the loop at 0.
// Stop reasons, per instance: 0 = max|g| <= gtol, 1 = max_iter iterations, 2 = no step of the
// line search lowered f (the point stays at the last accepted one). These are the rules of the
// host BFGS (qvs_bfgs_minimize), applied to every instance independently.
#include <math.h>
#include <string.h>

#include <vector>

#include "hc_batch.h"

namespace qvs {
namespace bopt {

constexpr int NT = 128;            // threads per step CTA; 2p <= 128 parameters per instance
constexpr int kMaxHalvings = 30;
constexpr double kC1 = 1e-4;

enum Stage : int { FIRST = 0, TRIAL = 1, DONE = 2 };

struct State {
  int m, th0;          // parameters (2p) and the offset of the instance's p layers
  int64_t voff, hoff;  // offsets of x, g, d (3m doubles) and H (m*m doubles)
  int stage, it, evals, halvings, stop;
  double f, a, slope;
};

struct StepArgs {
  State* st;
  double* vec;          // per instance: x[m], g[m], d[m]
  double* H;            // per instance: m*m, row-major
  double* gammas;       // b->theta (trial points in, results out)
  double* ts;
  const double* out_E;  // batched evaluation at the trial points
  const double* out_dg;
  const double* out_dt;
  int* active;
  int* nactive;
  double gtol;
  int max_iter;
};

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < NT / 32; ++w) s = fmax(s, red[w]);
  return s;
}

// The step's fp64 arithmetic is the host BFGS's (qvs_bfgs_minimize) operation for operation:
// products and sums rounded separately (no fused multiply-add), dot products summed in index order
// by one thread. Given the same objective values the two loops then take the same decisions.
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// sum_k a[k] b[k] in index order, by thread 0, broadcast through shared memory
__device__ __forceinline__ double ordered_dot(const double* a, const double* b, int m, double* bcast) {
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int k = 0; k < m; ++k) acc = dadd(acc, dmul(a[k], b[k]));
    *bcast = acc;
  }
  __syncthreads();
  return *bcast;
}

// theta component j of an instance: gamma_{j/2} (j even) or t_{j/2} (j odd)
__device__ __forceinline__ double& theta_ref(const StepArgs& a, int th0, int j) {
  return (j & 1) ? a.ts[th0 + (j >> 1)] : a.gammas[th0 + (j >> 1)];
}

__global__ void __launch_bounds__(NT) bfgs_step_kernel(const __grid_constant__ StepArgs A) {
  __shared__ double red[NT / 32];
  __shared__ double s_a[NT], s_b[NT], s_c[NT];
  __shared__ double s_dot;
  const int i = blockIdx.x, j = threadIdx.x;
  State& S = A.st[i];
  if (S.stage == DONE) return;
  const int m = S.m;
  const bool own = j < m;
  double* x = A.vec + S.voff;
  double* g = x + m;
  double* d = g + m;
  double* H = A.H + S.hoff;
  // the evaluation at the current trial point
  const double fE = A.out_E[i];
  const double gt = own ? ((j & 1) ? A.out_dt[S.th0 + (j >> 1)] : A.out_dg[S.th0 + (j >> 1)]) : 0.0;
  const double xt = own ? theta_ref(A, S.th0, j) : 0.0;
  const int stage = S.stage;
  bool direction = false;   // take a new search direction at the end
  int stop = -1;            // >= 0: the instance stops with this reason
  if (stage == FIRST) {
    if (own) {
      x[j] = xt;
      g[j] = gt;
      for (int k = 0; k < m; ++k) H[(size_t)j * m + k] = (k == j) ? 1.0 : 0.0;
    }
    const double gmax = block_max(own ? fabs(gt) : 0.0, red);
    if (gmax <= A.gtol) stop = 0;
    else if (A.max_iter <= 0) stop = 1;
    else direction = true;
    if (j == 0) {
      S.f = fE;
      S.evals = 1;
      S.it = 0;
    }
  } else {   // TRIAL
    const double f0 = S.f, a = S.a, slope = S.slope;
    if (fE <= dadd(f0, dmul(dmul(kC1, a), slope))) {
      // accept: s = x_t - x, y = g_t - g, inverse-Hessian update
      const double s = own ? dsub(xt, x[j]) : 0.0;
      const double y = own ? dsub(gt, g[j]) : 0.0;
      s_a[j] = y;
      s_b[j] = s;
      const double ys = ordered_dot(s_a, s_b, m, &s_dot);
      if (ys > 0.0) {
        double hy = 0.0;
        if (own)
          for (int k = 0; k < m; ++k) hy = dadd(hy, dmul(H[(size_t)j * m + k], s_a[k]));
        s_c[j] = hy;
        const double yHy = ordered_dot(s_a, s_c, m, &s_dot);
        const double rho = 1.0 / ys;
        const double cs = dadd(dmul(dmul(rho, rho), yHy), rho);
        if (own)
          for (int k = 0; k < m; ++k) {
            const double t1 = dadd(dmul(s_b[j], s_c[k]), dmul(s_c[j], s_b[k]));
            const double t2 = dadd(dmul(-rho, t1), dmul(dmul(cs, s_b[j]), s_b[k]));
            H[(size_t)j * m + k] = dadd(H[(size_t)j * m + k], t2);
          }
      }
      if (own) {
        x[j] = xt;
        g[j] = gt;
      }
      const double gmax = block_max(own ? fabs(gt) : 0.0, red);
      const int it = S.it + 1;
      if (gmax <= A.gtol) stop = 0;
      else if (it >= A.max_iter) stop = 1;
      else direction = true;
      __syncthreads();
      if (j == 0) {
        S.f = fE;
        S.it = it;
      }
    } else {
      const int h = S.halvings + 1;
      if (h > kMaxHalvings) {
        stop = 2;
      } else {
        __syncthreads();
        if (j == 0) {
          S.halvings = h;
          S.a = a * 0.5;
        }
        __syncthreads();
        if (own) theta_ref(A, S.th0, j) = dadd(x[j], dmul(S.a, d[j]));
      }
    }
    if (j == 0) S.evals += 1;
  }
  __syncthreads();
  if (direction) {
    s_a[j] = own ? g[j] : 0.0;
    __syncthreads();
    double acc = 0.0;
    if (own)
      for (int k = 0; k < m; ++k) acc = dadd(acc, dmul(H[(size_t)j * m + k], s_a[k]));
    s_b[j] = -acc;
    double slope = ordered_dot(s_a, s_b, m, &s_dot);
    if (slope >= 0.0) {   // not a descent direction: restart from steepest descent
      if (own)
        for (int k = 0; k < m; ++k) H[(size_t)j * m + k] = (k == j) ? 1.0 : 0.0;
      s_b[j] = -s_a[j];
      slope = ordered_dot(s_a, s_b, m, &s_dot);
    }
    if (own) {
      d[j] = s_b[j];
      theta_ref(A, S.th0, j) = dadd(x[j], dmul(1.0, s_b[j]));   // a = 1
    }
    if (j == 0) {
      S.slope = slope;
      S.a = 1.0;
      S.halvings = 0;
      S.stage = TRIAL;
    }
  }
  if (stop >= 0) {
    if (own) theta_ref(A, S.th0, j) = x[j];   // the result: the last accepted point
    if (j == 0) {
      S.stop = stop;
      S.stage = DONE;
      A.active[i] = 0;
    }
  } else if (j == 0) {
    A.active[i] = 1;
    atomicAdd(A.nactive, 1);
  }
}

}  // namespace bopt
}  // namespace qvs

using namespace qvs;

static int qvs_batch_optimise_impl(qvs_batch_t b, double* gammas, double* ts, double gtol, int max_iter,
                                   double* f_out, int* iters_out, int* evals_out, int* stop_out) {
  using bopt::State;
  if (!b || !gammas || !ts || max_iter < 0 || max_iter > 100000 || !(gtol >= 0.0)) return QVS_EINVAL;
  if (!b->have_q) return QVS_ESTATE;
  const int count = b->count;
  const size_t P = (size_t)b->total_p;
  for (size_t k = 0; k < P; ++k)
    if (!isfinite(gammas[k]) || !isfinite(ts[k])) return QVS_EINVAL;
  for (int i = 0; i < count; ++i)
    if (2 * b->p[i] > bopt::NT) return QVS_EUNSUPPORTED;
  // per-instance state and the vector / matrix pools
  std::vector<State> st(count);
  int64_t voff = 0, hoff = 0;
  for (int i = 0; i < count; ++i) {
    State& S = st[i];
    memset(&S, 0, sizeof(S));
    S.m = 2 * b->p[i];
    S.th0 = b->th0[i];
    S.voff = voff;
    S.hoff = hoff;
    S.stage = bopt::FIRST;
    voff += 3 * (int64_t)S.m;
    hoff += (int64_t)S.m * S.m;
  }
  QVS_TRY(b->opt_state.ensure(sizeof(State) * count));
  QVS_TRY(b->opt_vec.ensure(sizeof(double) * (size_t)voff));
  QVS_TRY(b->opt_H.ensure(sizeof(double) * (size_t)hoff));
  QVS_TRY(b->opt_active.ensure(sizeof(int) * count));
  QVS_TRY(b->opt_nactive.ensure(sizeof(int)));
  if (!b->host_nactive) QVS_CUDA_TRY(cudaMallocHost((void**)&b->host_nactive, sizeof(int)));
  cudaStream_t s = b->stream;
  QVS_CUDA_TRY(cudaMemcpyAsync(b->opt_state.ptr, st.data(), sizeof(State) * count, cudaMemcpyHostToDevice, s));
  std::vector<int> ones(count, 1);
  QVS_CUDA_TRY(cudaMemcpyAsync(b->opt_active.ptr, ones.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
  memcpy(b->host_theta, gammas, sizeof(double) * P);
  memcpy(b->host_theta + P, ts, sizeof(double) * P);
  QVS_CUDA_TRY(cudaMemcpyAsync(b->theta.ptr, b->host_theta, sizeof(double) * 2 * P, cudaMemcpyHostToDevice, s));
  QVS_TRY(hc::batch_autotune(b));   // times two launches at the start point on the first use

  bopt::StepArgs A{};
  A.st = b->opt_state.as<State>();
  A.vec = b->opt_vec.as<double>();
  A.H = b->opt_H.as<double>();
  A.gammas = b->theta.as<double>();
  A.ts = A.gammas + P;
  A.out_E = b->out.as<double>();
  A.out_dg = A.out_E + count;
  A.out_dt = A.out_dg + P;
  A.active = b->opt_active.as<int>();
  A.nactive = b->opt_nactive.as<int>();
  A.gtol = gtol;
  A.max_iter = max_iter;

  // one iteration (evaluate, step, count) as a graph; the buffers it names are fixed until the
  // batch is destroyed or its quality buffer moves, but gtol and max_iter change per call
  if (b->opt_graph) {
    cudaGraphExecDestroy(b->opt_graph);
    b->opt_graph = nullptr;
  }
  {
    cudaStream_t cs;
    QVS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    const cudaStream_t keep = b->stream;
    b->stream = cs;
    int stc = QVS_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) stc = QVS_ECUDA;
    if (stc == QVS_OK && cudaMemsetAsync(A.nactive, 0, sizeof(int), cs) != cudaSuccess) stc = QVS_ECUDA;
    if (stc == QVS_OK) stc = hc::batch_launch(b, b->ctas_per_sm, A.active);
    if (stc == QVS_OK) {
      bopt::bfgs_step_kernel<<<count, bopt::NT, 0, cs>>>(A);
      if (cudaGetLastError() != cudaSuccess) stc = QVS_ECUDA;
    }
    if (stc == QVS_OK &&
        cudaMemcpyAsync(b->host_nactive, A.nactive, sizeof(int), cudaMemcpyDeviceToHost, cs) != cudaSuccess)
      stc = QVS_ECUDA;
    const cudaError_t ce = cudaStreamEndCapture(cs, &g);
    b->stream = keep;
    cudaStreamDestroy(cs);
    if (stc != QVS_OK || ce != cudaSuccess) {   // a failed capture leaves no graph behind
      if (ce == cudaSuccess && g) cudaGraphDestroy(g);
      (void)cudaGetLastError();
      return stc != QVS_OK ? stc : QVS_ECUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->opt_graph, g, 0);
    cudaGraphDestroy(g);
    QVS_CUDA_TRY(ie);
  }
  QVS_CUDA_TRY(cudaStreamSynchronize(s));
  // each instance stops within max_iter * (kMaxHalvings + 1) + 1 evaluations
  const int64_t cap = (int64_t)max_iter * (bopt::kMaxHalvings + 1) + 1;
  for (int64_t r = 0; r < cap; ++r) {
    QVS_CUDA_TRY(cudaGraphLaunch(b->opt_graph, s));
    QVS_CUDA_TRY(cudaStreamSynchronize(s));
    if (*b->host_nactive == 0) break;
  }
  if (*b->host_nactive != 0) return QVS_ENUMERIC;
  QVS_CUDA_TRY(cudaMemcpyAsync(b->host_theta, b->theta.ptr, sizeof(double) * 2 * P, cudaMemcpyDeviceToHost, s));
  QVS_CUDA_TRY(cudaMemcpyAsync(st.data(), b->opt_state.ptr, sizeof(State) * count, cudaMemcpyDeviceToHost, s));
  QVS_CUDA_TRY(cudaStreamSynchronize(s));
  memcpy(gammas, b->host_theta, sizeof(double) * P);
  memcpy(ts, b->host_theta + P, sizeof(double) * P);
  for (int i = 0; i < count; ++i) {
    if (f_out) f_out[i] = st[i].f;
    if (iters_out) iters_out[i] = st[i].it;
    if (evals_out) evals_out[i] = st[i].evals;
    if (stop_out) stop_out[i] = st[i].stop;
  }
  return QVS_OK;
}

extern "C" int qvs_batch_optimise(qvs_batch_t b, double* gammas, double* ts, double gtol, int max_iter,
                                  double* f_out, int* iters_out, int* evals_out, int* stop_out) {
  return qvs::guarded([&] {
    return qvs_batch_optimise_impl(b, gammas, ts, gtol, max_iter, f_out, iters_out, evals_out, stop_out);
  });
}

// Sec. 5 (benchmark with param_persist): a depth sweep of repeated optimisations of one instance.
// Each depth is one batch of `repeats` parameter sets sharing the instance's qualities, optimised
// together; the best optimum of a depth seeds the first layers of every repeat at the next depth.
static int qvs_benchmark_impl(int n, const float* q, int on_device, int d_min, int d_max, int repeats,
                              const double* init, double gtol, int max_iter, double* f_out, double* best_theta,
                              void* stream) {
  if (!q || !init || !f_out || !best_theta || n < 12 || n > 28 || repeats < 1 || repeats > 65536 ||
      d_min < 1 || d_max < d_min || d_max > bopt::NT / 2 || max_iter < 0 || !(gtol >= 0.0))
    return QVS_EINVAL;
  std::vector<double> best_g, best_t;   // best optimum of the previous depth
  const double* next = init;
  double* fo = f_out;
  double* bo = best_theta;
  for (int D = d_min; D <= d_max; ++D) {
    std::vector<int32_t> ns(repeats, n), ps(repeats, D);
    std::vector<double> g((size_t)repeats * D), t((size_t)repeats * D);
    for (int r = 0; r < repeats; ++r) {
      if (D == d_min) {   // repeat r: gamma_1..gamma_D then t_1..t_D
        for (int k = 0; k < D; ++k) {
          g[(size_t)r * D + k] = next[(size_t)r * 2 * D + k];
          t[(size_t)r * D + k] = next[(size_t)r * 2 * D + D + k];
        }
      } else {            // persisted layers, then the repeat's own new layer
        for (int k = 0; k < D - 1; ++k) {
          g[(size_t)r * D + k] = best_g[k];
          t[(size_t)r * D + k] = best_t[k];
        }
        g[(size_t)r * D + D - 1] = next[2 * (size_t)r];
        t[(size_t)r * D + D - 1] = next[2 * (size_t)r + 1];
      }
    }
    next += D == d_min ? (size_t)repeats * 2 * D : (size_t)repeats * 2;
    qvs_batch_t b = nullptr;
    QVS_TRY(qvs_batch_create(&b, repeats, ns.data(), ps.data(), stream));
    int st = qvs_batch_set_quality_shared(b, q, on_device);
    if (st == QVS_OK) st = qvs_batch_optimise(b, g.data(), t.data(), gtol, max_iter, fo, nullptr, nullptr, nullptr);
    qvs_batch_destroy(b);
    if (st != QVS_OK) return st;
    int rb = 0;
    for (int r = 1; r < repeats; ++r)
      if (fo[r] < fo[rb]) rb = r;
    best_g.assign(g.begin() + (size_t)rb * D, g.begin() + (size_t)rb * D + D);
    best_t.assign(t.begin() + (size_t)rb * D, t.begin() + (size_t)rb * D + D);
    for (int k = 0; k < D; ++k) {
      bo[k] = best_g[k];
      bo[D + k] = best_t[k];
    }
    fo += repeats;
    bo += 2 * D;
  }
  return QVS_OK;
}

extern "C" int qvs_benchmark(int n, const float* q, int on_device, int d_min, int d_max, int repeats,
                             const double* init, double gtol, int max_iter, double* f_out, double* best_theta,
                             void* stream) {
  return qvs::guarded([&] {
    return qvs_benchmark_impl(n, q, on_device, d_min, d_max, repeats, init, gtol, max_iter, f_out, best_theta, stream);
  });
}
