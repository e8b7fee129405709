// Stencil step instantiations for radius R = 7 (space order 14).
#include "step_launch.cuh"
WAVE_DEFINE_STEP_RADIUS(7)
