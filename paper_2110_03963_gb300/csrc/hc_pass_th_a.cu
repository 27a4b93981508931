// complex64 tiled-pass kernels of the QAOA hypercube path for rotation thresholds 0, 2, 3
// (-1 = runtime masks); one translation unit per few thresholds keeps the build parallel.
#define QVS_HC_PASS_TU
#include "hc_staged.cuh"

namespace qvs {
namespace hc {

template int launch_pass<float, 0>(int, const PassArgs<float>&, uint32_t, cudaStream_t);
template int launch_pass<float, 2>(int, const PassArgs<float>&, uint32_t, cudaStream_t);
template int launch_pass<float, 3>(int, const PassArgs<float>&, uint32_t, cudaStream_t);

template int launch_staged<0>(int, const PassArgs<float>&, const StageMaps&, uint32_t, uint32_t, cudaStream_t);
template int launch_staged<2>(int, const PassArgs<float>&, const StageMaps&, uint32_t, uint32_t, cudaStream_t);
template int launch_staged<3>(int, const PassArgs<float>&, const StageMaps&, uint32_t, uint32_t, cudaStream_t);

}  // namespace hc
}  // namespace qvs
