// Explicit instantiation of the flash launch sequences for NC = 12.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(12)
}  // namespace ptf
