// Explicit instantiation of the flash launch sequences for NC = 7.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(7)
}  // namespace ptf
