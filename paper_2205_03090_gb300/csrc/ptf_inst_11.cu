// Explicit instantiation of the flash launch sequences for NC = 11.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(11)
}  // namespace ptf
