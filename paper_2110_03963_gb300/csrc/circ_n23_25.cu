// Circulant (QWOA) path, column transform geometries (N = 2^23: Geo<5, 3, 3, 3>, N = 2^25: Geo<3, 3, 4, 4>).
#include "circ_impl.cuh"

namespace qvs {
namespace cf {

int set_mixer_n23(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs) {
  return Driver<Geo<5, 3, 3, 3>>::set_mixer(h, ofs, w, nofs);
}

int run_n23(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt) {
  return Driver<Geo<5, 3, 3, 3>>::run(h, p, gammas, ts, grad, E, dg, dt);
}

int set_mixer_n25(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs) {
  return Driver<Geo<3, 3, 4, 4>>::set_mixer(h, ofs, w, nofs);
}

int run_n25(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt) {
  return Driver<Geo<3, 3, 4, 4>>::run(h, p, gammas, ts, grad, E, dg, dt);
}

}  // namespace cf
}  // namespace qvs
