// Circulant (QWOA) path for N = 2^24: instantiation of the column transform geometry Geo<4, 3, 3, 4>.
#include "circ_impl.cuh"

namespace qvs {
namespace cf {

int set_mixer_n24(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs) {
  return Driver<Geo<4, 3, 3, 4>>::set_mixer(h, ofs, w, nofs);
}

int run_n24(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt) {
  return Driver<Geo<4, 3, 3, 4>>::run(h, p, gammas, ts, grad, E, dg, dt);
}

}  // namespace cf
}  // namespace qvs
