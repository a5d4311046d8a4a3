// Kernels for window radius 6.
#define OF_RADIUS 6
#include "radius_impl.cuh"
