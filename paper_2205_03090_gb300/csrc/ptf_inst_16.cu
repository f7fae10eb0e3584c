// Explicit instantiation of the flash launch sequences for NC = 16.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(16)
}  // namespace ptf
