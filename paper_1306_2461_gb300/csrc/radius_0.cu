// Kernels for window radius 0 (0: any radius, given at run time).
#define OF_RADIUS 0
#include "radius_impl.cuh"
