// Mixed-precision echo path, variant 2 (u-v antenna gain grids).
#define HARM_MIXED_VARIANT 2
#include "echo_mixed.cuh"
