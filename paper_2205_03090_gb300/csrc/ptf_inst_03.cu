// Explicit instantiation of the flash launch sequences for NC = 3.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(3)
}  // namespace ptf
