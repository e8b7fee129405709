// Stencil step instantiations for radius R = 3 (space order 6).
#include "step_launch.cuh"
WAVE_DEFINE_STEP_RADIUS(3)
