// Explicit instantiation of the flash launch sequences for NC = 2.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(2)
}  // namespace ptf
