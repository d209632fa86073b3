// Order-3 MHD predictor + face kernel in F32 (see step_inst.cuh).
#define ADER_ORDER 3
#define ADER_NV 8
#define ADER_REAL float
#include "step_inst.cuh"
