// Mixed-precision echo path, variant 3 (Choppy Wave Model with u-v antenna gain grids).
#define HARM_MIXED_VARIANT 3
#include "echo_mixed.cuh"
