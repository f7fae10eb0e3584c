// Explicit instantiation of the flash launch sequences for NC = 13.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(13)
}  // namespace ptf
