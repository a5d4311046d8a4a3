// Kernels for window radius 8.
#define OF_RADIUS 8
#include "radius_impl.cuh"
