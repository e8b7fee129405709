// Stencil step instantiations for radius R = 2 (space order 4).
#include "step_launch.cuh"
WAVE_DEFINE_STEP_RADIUS(2)
