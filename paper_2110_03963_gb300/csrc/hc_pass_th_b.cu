// complex64 tiled-pass kernels of the QAOA hypercube path for rotation thresholds 4, 5, 6
// (-1 = runtime masks); one translation unit per few thresholds keeps the build parallel.
#define QVS_HC_PASS_TU
#include "hc_staged.cuh"

namespace qvs {
namespace hc {

template int launch_pass<float, 4>(int, const PassArgs<float>&, uint32_t, cudaStream_t);
template int launch_pass<float, 5>(int, const PassArgs<float>&, uint32_t, cudaStream_t);
template int launch_pass<float, 6>(int, const PassArgs<float>&, uint32_t, cudaStream_t);

template int launch_staged<4>(int, const PassArgs<float>&, const StageMaps&, uint32_t, uint32_t, cudaStream_t);
template int launch_staged<5>(int, const PassArgs<float>&, const StageMaps&, uint32_t, uint32_t, cudaStream_t);
template int launch_staged<6>(int, const PassArgs<float>&, const StageMaps&, uint32_t, uint32_t, cudaStream_t);

}  // namespace hc
}  // namespace qvs
