// Launchers of the float32 Born kernels (all supported axis extents).
#include "launch.cuh"
namespace cbs {
CBS_INSTANTIATE_LAUNCHERS(float)
}
