// Explicit instantiation of the flash launch sequences for NC = 8.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(8)
}  // namespace ptf
