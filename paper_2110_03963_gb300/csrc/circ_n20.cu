// Circulant (QWOA) path for N = 2^20: instantiation of the column transform geometry Geo<8, 2, 2, 2>.
#include "circ_impl.cuh"

namespace qvs {
namespace cf {

int set_mixer_n20(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs) {
  return Driver<Geo<8, 2, 2, 2>>::set_mixer(h, ofs, w, nofs);
}

int run_n20(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt) {
  return Driver<Geo<8, 2, 2, 2>>::run(h, p, gammas, ts, grad, E, dg, dt);
}

}  // namespace cf
}  // namespace qvs
