// Stencil step instantiations for radius R = 1 (space order 2).
#include "step_launch.cuh"
WAVE_DEFINE_STEP_RADIUS(1)
