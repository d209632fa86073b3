// Order-4 MHD predictor + face kernel in F32 (see step_inst.cuh).
#define ADER_ORDER 4
#define ADER_NV 8
#define ADER_REAL float
#include "step_inst.cuh"
