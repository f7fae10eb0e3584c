// Explicit instantiation of the flash launch sequences for NC in {9 10 11}.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
template cudaError_t launch_plain<9>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
template cudaError_t launch_plain<10>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
template cudaError_t launch_plain<11>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
}  // namespace ptf
