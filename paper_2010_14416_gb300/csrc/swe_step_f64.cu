// FP64 instantiation of the step kernels (IEEE division and square root).
#include "swe_launch.cuh"

namespace swe {
template struct Launch<double>;
}
