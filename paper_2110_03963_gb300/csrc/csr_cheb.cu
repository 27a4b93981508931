// QAOAz sparse-mixer path (Sec. 2.4.1, Sec. 3) - placeholder until the Chebyshev kernels land.
#include "qvs_internal.h"

namespace qvs {
int csr_set_mixer(qvs_ctx*, const qvs_mixer_desc*) { return QVS_EUNSUPPORTED; }
int csr_evolve(qvs_ctx*, int, const double*, const double*) { return QVS_EUNSUPPORTED; }
int csr_gradient(qvs_ctx*, int, const double*, const double*, double*, double*, double*) {
  return QVS_EUNSUPPORTED;
}
}  // namespace qvs
