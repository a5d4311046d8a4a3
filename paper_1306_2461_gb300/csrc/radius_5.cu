// Kernels for window radius 5.
#define OF_RADIUS 5
#include "radius_impl.cuh"
