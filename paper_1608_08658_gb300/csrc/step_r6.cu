// Stencil step instantiations for radius R = 6 (space order 12).
#include "step_launch.cuh"
WAVE_DEFINE_STEP_RADIUS(6)
