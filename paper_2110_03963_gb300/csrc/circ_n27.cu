// Circulant (QWOA) path, column transform geometries (N = 2^27: Geo<1, 4, 4, 5>).
#include "circ_impl.cuh"

namespace qvs {
namespace cf {

int set_mixer_n27(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs) {
  return Driver<Geo<1, 4, 4, 5>>::set_mixer(h, ofs, w, nofs);
}

int run_n27(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt) {
  return Driver<Geo<1, 4, 4, 5>>::run(h, p, gammas, ts, grad, E, dg, dt);
}

}  // namespace cf
}  // namespace qvs
