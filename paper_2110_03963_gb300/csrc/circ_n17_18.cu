// Circulant (QWOA) path, column transform geometries (N = 2^17: Geo<11, 1, 1, 1>, N = 2^18: Geo<10, 1, 1, 2>).
#include "circ_impl.cuh"

namespace qvs {
namespace cf {

int set_mixer_n17(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs) {
  return Driver<Geo<11, 1, 1, 1>>::set_mixer(h, ofs, w, nofs);
}

int run_n17(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt) {
  return Driver<Geo<11, 1, 1, 1>>::run(h, p, gammas, ts, grad, E, dg, dt);
}

int set_mixer_n18(qvs_ctx* h, const int64_t* ofs, const double* w, int nofs) {
  return Driver<Geo<10, 1, 1, 2>>::set_mixer(h, ofs, w, nofs);
}

int run_n18(qvs_ctx* h, int p, const double* gammas, const double* ts, bool grad, double* E, double* dg,
            double* dt) {
  return Driver<Geo<10, 1, 1, 2>>::run(h, p, gammas, ts, grad, E, dg, dt);
}

}  // namespace cf
}  // namespace qvs
