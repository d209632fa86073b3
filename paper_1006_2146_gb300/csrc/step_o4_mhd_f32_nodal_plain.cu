// Order-4 MHD predictor + face kernel in F32, nodal form, without a source (see step_inst.cuh).
#define ADER_ORDER 4
#define ADER_NV 8
#define ADER_REAL float
#define ADER_FORM FORM_NODAL
#define ADER_SRC false
#include "step_inst.cuh"
