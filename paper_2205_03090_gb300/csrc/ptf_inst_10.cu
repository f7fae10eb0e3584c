// Explicit instantiation of the flash launch sequences for NC = 10.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(10)
}  // namespace ptf
