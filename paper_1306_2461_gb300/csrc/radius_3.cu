// Kernels for window radius 3.
#define OF_RADIUS 3
#include "radius_impl.cuh"
