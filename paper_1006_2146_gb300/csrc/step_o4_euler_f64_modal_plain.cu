// Order-4 Euler predictor + face kernel in F64, modal form, without a source (see step_inst.cuh).
#define ADER_ORDER 4
#define ADER_NV 5
#define ADER_REAL double
#define ADER_FORM FORM_MODAL
#define ADER_SRC false
#include "step_inst.cuh"
