// Stencil step instantiations for radius R = 4 (space order 8).
#include "step_launch.cuh"
WAVE_DEFINE_STEP_RADIUS(4)
