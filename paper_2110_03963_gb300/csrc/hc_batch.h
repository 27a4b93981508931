// Host state of a batched solve (qvs_batch_*): shared by the batched gradient (hypercube.cu) and
// the batched optimiser (batch_opt.cu).
#pragma once

#include <string>
#include <vector>

#include "qvs_internal.h"

struct qvs_batch {
  int count = 0;
  int total_p = 0;
  int64_t total_q = 0;
  cudaStream_t stream = nullptr;
  std::vector<int> n, p, th0;
  std::vector<int64_t> qoff;
  qvs::DevBuf inst, order, q, theta, out, counter, ws;
  size_t slot_bytes = 0;
  int64_t dim_max = 0;
  int nck_max = 0;
  int nslots = 0;
  int sms = 0;
  int ctas_per_sm = 0;       // chosen by the autotuner on the first solve (0 = not yet tuned)
  double tuned_ms[3] = {0, 0, 0};
  // schedule candidates: checkpoint policy 0 = the forward state every ceil(sqrt(p)) layers
  // (uncompute in between), 1 = every pass boundary (no uncompute, more workspace)
  int ckpt_policy = 0;
  bool from_cache = false;
  double trial_ms4[4] = {0, 0, 0, 0};             // policy 0 at 1, 2 CTAs/SM, policy 1 at 1, 2
  std::vector<unsigned char> host_inst[2];         // instance tables per policy (host copies)
  size_t slot_bytes_pol[2] = {0, 0};
  int nck_max_pol[2] = {0, 0};
  double model_bytes_pol[2] = {0.0, 0.0};
  std::string gpu_name;
  double* host_theta = nullptr;   // pinned: gammas then ts
  double* host_out = nullptr;     // pinned: E, dg, dt
  cudaGraphExec_t graph = nullptr;
  bool have_q = false;
  bool shared_q = false;          // every instance reads the same 2^n qualities
  double model_bytes = 0.0, model_fma = 0.0, amp_layers = 0.0;   // cost model of one solve

  // batched BFGS (batch_opt.cu)
  qvs::DevBuf opt_state, opt_vec, opt_H, opt_active, opt_nactive;
  int64_t opt_vec_len = 0, opt_H_len = 0;
  cudaGraphExec_t opt_graph = nullptr;
  int* host_nactive = nullptr;    // pinned
};

namespace qvs {
namespace hc {
// One launch of the persistent batched kernel: objective and gradient of every instance at the
// parameters in b->theta, into b->out. active (device, count flags, or NULL = all): instances whose
// flag is 0 are skipped and their outputs left as they were.
int batch_launch(qvs_batch_t b, int ctas_per_sm, const int* active);
// Pick the schedule (first call only): from the schedule cache, else by timing one launch per
// candidate (CTAs per SM x checkpoint policy); needs b->theta set.
int batch_autotune(qvs_batch_t b);
// Switch to checkpoint policy pol (0: every ceil(sqrt(p)) layers, 1: every pass boundary).
int batch_configure(qvs_batch_t b, int pol);
}  // namespace hc
}  // namespace qvs
