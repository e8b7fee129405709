// Stencil step instantiations for radius R = 8 (space order 16).
#include "step_launch.cuh"
WAVE_DEFINE_STEP_RADIUS(8)
