// Explicit instantiation of the flash launch sequences for NC in {6 7 8}.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
template cudaError_t launch_plain<6>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
template cudaError_t launch_plain<7>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
template cudaError_t launch_plain<8>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
}  // namespace ptf
