// Order-4 Euler predictor + face kernel in F32, nodal form, with a source (see step_inst.cuh).
#define ADER_ORDER 4
#define ADER_NV 5
#define ADER_REAL float
#define ADER_FORM FORM_NODAL
#define ADER_SRC true
#include "step_inst.cuh"
