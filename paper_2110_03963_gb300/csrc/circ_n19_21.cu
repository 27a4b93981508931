// Circulant (QWOA) path, column transform geometries (N = 2^19: Geo<9, 1, 2, 2>, N = 2^21: Geo<7, 2, 2, 3>).
#include "circ_impl.cuh"

namespace qvs {
namespace cf {

int set_mixer_n19(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs) {
  return Driver<Geo<9, 1, 2, 2>>::set_mixer(h, ofs, w, nofs);
}

int run_n19(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt) {
  return Driver<Geo<9, 1, 2, 2>>::run(h, p, gammas, ts, grad, E, dg, dt);
}

int set_mixer_n21(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs) {
  return Driver<Geo<7, 2, 2, 3>>::set_mixer(h, ofs, w, nofs);
}

int run_n21(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt) {
  return Driver<Geo<7, 2, 2, 3>>::run(h, p, gammas, ts, grad, E, dg, dt);
}

}  // namespace cf
}  // namespace qvs
