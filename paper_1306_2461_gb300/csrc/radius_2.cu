// Kernels for window radius 2.
#define OF_RADIUS 2
#include "radius_impl.cuh"
