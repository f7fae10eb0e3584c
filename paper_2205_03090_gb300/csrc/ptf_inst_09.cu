// Explicit instantiation of the flash launch sequences for NC = 9.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(9)
}  // namespace ptf
