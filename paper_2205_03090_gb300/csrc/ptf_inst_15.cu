// Explicit instantiation of the flash launch sequences for NC = 15.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(15)
}  // namespace ptf
