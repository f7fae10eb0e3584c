// Explicit instantiation of the flash launch sequences for NC = 5.
#include <cmath>
#include "ptf_launch.cuh"
namespace ptf {
PTF_INSTANTIATE_NC(5)
}  // namespace ptf
