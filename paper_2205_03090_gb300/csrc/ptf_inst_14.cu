// Explicit instantiation of the flash launch sequences for NC = 14.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(14)
}  // namespace ptf
