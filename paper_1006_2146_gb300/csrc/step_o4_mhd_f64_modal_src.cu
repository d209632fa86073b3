// Order-4 MHD predictor + face kernel in F64, modal form, with a source (see step_inst.cuh).
#define ADER_ORDER 4
#define ADER_NV 8
#define ADER_REAL double
#define ADER_FORM FORM_MODAL
#define ADER_SRC true
#include "step_inst.cuh"
