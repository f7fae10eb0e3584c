// Explicit instantiation of the flash launch sequences for NC = 6.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(6)
}  // namespace ptf
