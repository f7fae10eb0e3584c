// Explicit instantiation of the flash launch sequences for NC in {2 3 4 5}.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
template cudaError_t launch_plain<2>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
template cudaError_t launch_plain<3>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
template cudaError_t launch_plain<4>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
template cudaError_t launch_plain<5>(const CompHost&, const WS&, const IO&, int, int, cudaStream_t, cudaEvent_t*, const MLP*, float,
                                   float);
}  // namespace ptf
