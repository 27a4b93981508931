// QWOA circulant-mixer path (Sec. 2.4.2, Sec. 3): exp(-i t W) = F^-1 exp(-i t Lambda) F.
//
// Passes over a state of N = 2^n amplitudes (n = 14 + B), each a tile of 2^14 amplitudes:
//   column pass: tile = 2^(14-B) adjacent columns x 2^B rows (index bits 14..n-1); it finishes the
//                inverse column transform of layer k, applies the phase of layer k+1 and starts
//                the column transform of layer k+1 (with the four-step twiddle omega_N^(j_low k_col));
//   row pass:    tile = 2^14 contiguous amplitudes; row transform, eigenphase exp(-i t lambda_k),
//                inverse row transform.
// A layer costs two passes (p+1 column passes and p row passes in total).
//
// Gradient: every column pass stores psi_k (natural basis) and every row pass stores the Fourier
// coefficients of psi_k, each in a private thread-major order. The adjoint sweep then moves only
// lambda through the inverse passes and reads those stored vectors for the two inner products
//   df/dt_k     = 2/N Im sum_k conj(F lambda)_k lambda_k (F psi_k)_k   (row pass)
//   df/dgamma_k = 2 Im <lambda|Q P_k psi_{k-1}>                        (column pass)
// so no state is uncomputed.
#include <math.h>

#include <vector>

#include "fft_kernels.cuh"
#include "qvs_internal.h"

namespace qvs {
namespace cf {

int set_mixer_n17(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs);
int run_n17(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt);
int set_mixer_n18(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs);
int run_n18(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt);
int set_mixer_n19(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs);
int run_n19(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt);
int set_mixer_n20(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs);
int run_n20(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt);
int set_mixer_n21(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs);
int run_n21(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt);
int set_mixer_n22(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs);
int run_n22(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt);
int set_mixer_n23(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs);
int run_n23(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt);
int set_mixer_n24(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs);
int run_n24(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt);
int set_mixer_n25(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs);
int run_n25(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt);
int set_mixer_n26(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs);
int run_n26(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt);
int set_mixer_n27(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs);
int run_n27(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt);

static int dispatch_set_mixer(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs) {
  switch (h->n) {
    case 17: return set_mixer_n17(h, ofs, w, nofs);
    case 18: return set_mixer_n18(h, ofs, w, nofs);
    case 19: return set_mixer_n19(h, ofs, w, nofs);
    case 20: return set_mixer_n20(h, ofs, w, nofs);
    case 21: return set_mixer_n21(h, ofs, w, nofs);
    case 22: return set_mixer_n22(h, ofs, w, nofs);
    case 23: return set_mixer_n23(h, ofs, w, nofs);
    case 24: return set_mixer_n24(h, ofs, w, nofs);
    case 25: return set_mixer_n25(h, ofs, w, nofs);
    case 26: return set_mixer_n26(h, ofs, w, nofs);
    case 27: return set_mixer_n27(h, ofs, w, nofs);
  }
  return QVS_EUNSUPPORTED;
}

static int dispatch_run(qvs_ctx* h, int p, const double* g, const double* t, bool grad, double* E, double* dg,
                        double* dt) {
  switch (h->n) {
    case 17: return run_n17(h, p, g, t, grad, E, dg, dt);
    case 18: return run_n18(h, p, g, t, grad, E, dg, dt);
    case 19: return run_n19(h, p, g, t, grad, E, dg, dt);
    case 20: return run_n20(h, p, g, t, grad, E, dg, dt);
    case 21: return run_n21(h, p, g, t, grad, E, dg, dt);
    case 22: return run_n22(h, p, g, t, grad, E, dg, dt);
    case 23: return run_n23(h, p, g, t, grad, E, dg, dt);
    case 24: return run_n24(h, p, g, t, grad, E, dg, dt);
    case 25: return run_n25(h, p, g, t, grad, E, dg, dt);
    case 26: return run_n26(h, p, g, t, grad, E, dg, dt);
    case 27: return run_n27(h, p, g, t, grad, E, dg, dt);
  }
  return QVS_EUNSUPPORTED;
}

}  // namespace cf

int circ_set_mixer(qvs_ctx* h, const qvs_mixer_desc* d) {
  using namespace cf;
  if (h->precision != QVS_C64) return QVS_EUNSUPPORTED;
  if (h->n < 0) return QVS_EINVAL;
  if (d->n_offsets < 1 || d->n_offsets > 4096 || !d->offsets) return QVS_EINVAL;
  const int64_t N = h->dim;
  for (int i = 0; i < d->n_offsets; ++i) {
    if (d->offsets[i] <= 0 || d->offsets[i] >= N) return QVS_EINVAL;
    if (d->offset_weights && !isfinite(d->offset_weights[i])) return QVS_EINVAL;
  }
  std::vector<double> wt(d->n_offsets, 1.0);
  if (d->offset_weights)
    for (int i = 0; i < d->n_offsets; ++i) wt[i] = d->offset_weights[i];
  QVS_TRY(h->work.ensure(sizeof(int64_t) * d->n_offsets + sizeof(double) * d->n_offsets));
  int64_t* ofs_dev = h->work.as<int64_t>();
  double* w_dev = reinterpret_cast<double*>(ofs_dev + d->n_offsets);
  QVS_CUDA_TRY(cudaMemcpyAsync(ofs_dev, d->offsets, sizeof(int64_t) * d->n_offsets, cudaMemcpyHostToDevice,
                               h->stream));
  QVS_CUDA_TRY(cudaMemcpyAsync(w_dev, wt.data(), sizeof(double) * d->n_offsets, cudaMemcpyHostToDevice,
                               h->stream));
  const int st = dispatch_set_mixer(h, ofs_dev, w_dev, d->n_offsets);
  if (st != QVS_OK) return st;
  QVS_CUDA_TRY(cudaStreamSynchronize(h->stream));   // host staging buffers go out of scope
  h->circ.qT_valid = false;
  return QVS_OK;
}

int circ_evolve(qvs_ctx* h, int p, const double* gammas, const double* ts) {
  double E = 0.0;
  const int st = cf::dispatch_run(h, p, gammas, ts, false, &E, nullptr, nullptr);
  if (st != QVS_OK) return st;
  h->E = E;
  h->have_E = true;
  return QVS_OK;
}

int circ_gradient(qvs_ctx* h, int p, const double* gammas, const double* ts, double* E, double* dg,
                  double* dt) {
  return cf::dispatch_run(h, p, gammas, ts, true, E, dg, dt);
}

}  // namespace qvs
