// Explicit instantiation of the flash launch sequences for NC = 4.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(4)
}  // namespace ptf
