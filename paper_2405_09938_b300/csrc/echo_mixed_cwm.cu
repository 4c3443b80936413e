// Mixed-precision echo path, variant 1 (Choppy Wave Model).
#define HARM_MIXED_VARIANT 1
#include "echo_mixed.cuh"
