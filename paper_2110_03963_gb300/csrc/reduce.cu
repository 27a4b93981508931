// Deterministic fp64 reduction of per-CTA partial sums (objective and gradient components).
#include "qvs_internal.h"

namespace qvs {

__global__ void __launch_bounds__(256) reduce_rows_kernel(const double* __restrict__ part,
                                                          int64_t nblk, const int* __restrict__ rowmap,
                                                          double* __restrict__ out) {
  __shared__ double red[8];
  const int slot = blockIdx.x;
  double s = 0.0;
  for (int k = 0; k < 3; ++k) {
    const int row = rowmap[3 * slot + k];
    if (row < 0) continue;
    const double* pr = part + (size_t)row * nblk;
    for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) s += pr[b];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    out[slot] = t;
  }
}

int reduce_rows(qvs_ctx* h, const double* part, int64_t nblk, const int* rowmap_dev, int nslots,
                double* out_dev) {
  reduce_rows_kernel<<<nslots, 256, 0, h->stream>>>(part, nblk, rowmap_dev, out_dev);
  QVS_CUDA_TRY(cudaGetLastError());
  return QVS_OK;
}

}  // namespace qvs
