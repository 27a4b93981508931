// Circulant (QWOA) path for N = 2^22: instantiation of the column transform geometry Geo<6, 2, 3, 3>.
#include "circ_impl.cuh"

namespace qvs {
namespace cf {

int set_mixer_n22(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs) {
  return Driver<Geo<6, 2, 3, 3>>::set_mixer(h, ofs, w, nofs);
}

int run_n22(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt) {
  return Driver<Geo<6, 2, 3, 3>>::run(h, p, gammas, ts, grad, E, dg, dt);
}

}  // namespace cf
}  // namespace qvs
