// Explicit instantiation of the flash launch sequences for NC in {12 13}.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
template cudaError_t launch_plain<12>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
template cudaError_t launch_plain<13>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
}  // namespace ptf
