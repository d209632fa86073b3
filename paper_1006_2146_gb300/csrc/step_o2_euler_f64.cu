// Order-2 Euler predictor + face kernel in F64 (see step_inst.cuh).
#define ADER_ORDER 2
#define ADER_NV 5
#define ADER_REAL double
#include "step_inst.cuh"
