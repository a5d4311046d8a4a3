// Kernels for window radius 10.
#define OF_RADIUS 10
#include "radius_impl.cuh"
