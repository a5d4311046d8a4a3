// Kernels for window radius 4.
#define OF_RADIUS 4
#include "radius_impl.cuh"
