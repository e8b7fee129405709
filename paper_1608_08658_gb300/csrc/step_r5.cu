// Stencil step instantiations for radius R = 5 (space order 10).
#include "step_launch.cuh"
WAVE_DEFINE_STEP_RADIUS(5)
