// Explicit instantiation of the flash launch sequences for NC in {14 15 16}.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
template cudaError_t launch_plain<14>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
template cudaError_t launch_plain<15>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
template cudaError_t launch_plain<16>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
}  // namespace ptf
