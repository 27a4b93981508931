// QWOA circulant-mixer path (Sec. 2.4.2, Sec. 3) - placeholder until the FFT passes land.
#include "qvs_internal.h"

namespace qvs {
int circ_set_mixer(qvs_ctx*, const qvs_mixer_desc*) { return QVS_EUNSUPPORTED; }
int circ_evolve(qvs_ctx*, int, const double*, const double*) { return QVS_EUNSUPPORTED; }
int circ_gradient(qvs_ctx*, int, const double*, const double*, double*, double*, double*) {
  return QVS_EUNSUPPORTED;
}
}  // namespace qvs
